// mmsar_image_static: the imaging call for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc once they are running: a hard
// real-time acquisition loop that forbids any call that may block, fail on
// fragmentation or synchronise the device after start-up; a plug-in whose
// host application hands it only streams and the buffers it owns; firmware
// style deployments that fix their memory map when they boot.  They still
// own their inputs and output, but cannot provide the scratch workspace that
// mmsar_image needs.  This entry point runs the same launch sequence as
// mmsar_image on a scratch area that is part of the library image itself: a
// file-scope __device__ array of kStaticWsBytes.  Every GPU on which the
// library is used holds that array from module load until the process exits.
//
// In host code the array's name is only a host-side stand-in, so the device
// address is looked up with cudaGetSymbolAddress while the device is
// current.  A call made outside stream capture looks it up afresh (a device
// reset reloads the module, and the array may then sit elsewhere) and
// remembers it for its device; a call made while its stream is being
// captured cannot do that lookup and uses the address remembered by the last
// plain call on the device, so make one plain call on each device before any
// stream capture (and again after a device reset).  All calls on a device
// share the one array: calls whose work overlaps on the GPU (two streams, or
// two threads) race on it and must be serialised by the caller.  The array
// keeps the previous call's contents; mmsar_image clears the parts that must
// start at zero (error word, bin counters) at the start of every call and
// overwrites everything else it reads.  The error word sits at the start of
// the array: mmsar_poll_error(NULL, stream) reads it.
#include <mutex>

#include "internal.cuh"

namespace mmsar {

constexpr size_t kStaticWsBytes = 32ull << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_static_workspace[kStaticWsBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
}  // namespace

mmsar_status static_workspace_address(cudaStream_t s, void **out) {
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(MMSAR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return report_error(MMSAR_ERR_UNSUPPORTED_SIZE, "device %d beyond the %d supported", dev, kMaxDevices);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // not sticky; treat the stream as capturing
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess || !p)
            return report_error(MMSAR_ERR_CUDA, "looking up the static scratch area: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return report_error(MMSAR_ERR_INVALID_ARG,
                            "mmsar_image_static under stream capture needs one plain call on device %d first "
                            "(to look up its scratch area)", dev);
    }
    *out = g_addr[dev];
    return MMSAR_OK;
}

}  // namespace mmsar

using namespace mmsar;

extern "C" size_t mmsar_static_workspace_bytes(void) { return kStaticWsBytes; }

extern "C" mmsar_status mmsar_image_static(mmsar_plan *plan, const void *echo, const float *echo_scale,
                                           const double *pos, const double *tx, const double *rx, void *vol,
                                           void *stream) {
    if (!plan) return report_error(MMSAR_ERR_INVALID_ARG, "null plan");
    if (plan->p.ws_bytes > kStaticWsBytes)
        return report_error(MMSAR_ERR_UNSUPPORTED_SIZE,
                            "this scan needs %zu bytes of scratch; the built-in scratch area of "
                            "mmsar_image_static holds %zu bytes (use mmsar_image with a workspace)",
                            plan->p.ws_bytes, kStaticWsBytes);
    void *ws = nullptr;
    const mmsar_status st = static_workspace_address(reinterpret_cast<cudaStream_t>(stream), &ws);
    if (st != MMSAR_OK) return st;
    return mmsar_image(plan, ws, kStaticWsBytes, echo, echo_scale, pos, tx, rx, vol, stream);
}
