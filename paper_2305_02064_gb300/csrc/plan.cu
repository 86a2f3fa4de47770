// C ABI of libmmsar: plan creation and validation, workspace layout and the
// launch sequence of one image (see include/mmsar.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "internal.cuh"

namespace mmsar {

static thread_local std::string g_last_error;

static mmsar_status fail(mmsar_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

mmsar_status report_error(mmsar_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

static mmsar_status cuda_fail(cudaError_t e, const char *where) {
    return fail(MMSAR_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Relative L2 error of one Gaussian-gridding transform at oversampling 2
// with the Greengard-Lee tau, measured against the direct sum for kernel
// widths 4..12 (random points, 64 modes).  The plan picks the smallest
// width whose error is within the requested tolerance.
static const double kGaussErr[13] = {0, 0, 0, 0, 4.8e-3, 1.4e-3, 5.5e-4, 1.5e-4, 5.4e-5, 1.6e-5, 4.4e-6,
                                     1.3e-6, 3.5e-7};

// ------------------------------------------------------------------ fused header clear
// The region of each workspace that a new image must find zero (header,
// z_ref partial sums, bin counts): 16-byte stores.
struct ClearArgs {
    int4 *p;
    long long n16;
};

__global__ void __launch_bounds__(256) clear_multi(const __grid_constant__ BatchTable<ClearArgs> t) {
    int bid, nb;
    const ClearArgs &c = t.a[batch_scan(t, bid, nb)];
    int4 *p = c.p;
    const long long n16 = c.n16;
    for (long long i = (long long)bid * 256 + threadIdx.x; i < n16; i += (long long)nb * 256)
        p[i] = make_int4(0, 0, 0, 0);
}

cudaError_t launch_clear_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<ClearArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        const Plan &p = r[i].plan->p;
        const size_t bytes = p.off_counts + sizeof(int) * (size_t)p.n_bins;   // a multiple of 16
        args[i].p = reinterpret_cast<int4 *>(r[i].workspace);
        args[i].n16 = (long long)(bytes / 16);
        blocks[i] = (int)std::min<long long>((args[i].n16 + 1023) / 1024, 1024);
    }
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int, const BatchTable<ClearArgs> &t, int total) {
                             clear_multi<<<total, 256, 0, s>>>(t);
                             return cudaGetLastError();
                         });
}

static int width_for_tol(double tol) {
    for (int w = 4; w <= 12; ++w)
        if (kGaussErr[w] <= tol) return w;
    return 12;
}

cudaError_t ensure_smem_attr(const void *func, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    // The attribute is per device and per kernel; remember the largest value
    // set for each (kernel, device) and raise it when a launch needs more.
    struct Entry { const void *f; int dev; size_t bytes; };
    static Entry table[256];
    static int used = 0;
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    Entry *hit = nullptr;
    for (int i = 0; i < used; ++i)
        if (table[i].f == func && table[i].dev == dev) hit = &table[i];
    if (hit && hit->bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (hit)
        hit->bytes = bytes;
    else if (used < 256)
        table[used++] = Entry{func, dev, bytes};
    return cudaSuccess;
}

static mmsar_status build_plan(Plan &p, const mmsar_shape &sh, const mmsar_grid &g, const mmsar_options &o) {
    p.shape = sh;
    p.grid = g;
    p.opt = o;
    if (sh.n_tx < 1 || sh.n_rx < 1 || sh.n_pos < 0)
        return fail(MMSAR_ERR_INVALID_ARG, "n_tx, n_rx must be >= 1 and n_pos >= 0 (got %d, %d, %d)", sh.n_tx,
                    sh.n_rx, sh.n_pos);
    if (sh.n_k < 1 || sh.n_k > kMaxNk)
        return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "n_k must be in 1..%d (got %d)", kMaxNk, sh.n_k);
    if (!(sh.f0_hz > 0.0) || !std::isfinite(sh.f0_hz) || (sh.n_k > 1 && !(sh.df_hz > 0.0)) ||
        !std::isfinite(sh.df_hz))
        return fail(MMSAR_ERR_INVALID_ARG, "f0_hz must be > 0 and df_hz > 0");
    if (sh.dtype != MMSAR_ECHO_C64 && sh.dtype != MMSAR_ECHO_F16X2_SCALED && sh.dtype != MMSAR_ECHO_BF16X2_SCALED)
        return fail(MMSAR_ERR_INVALID_ARG, "unknown echo dtype %d", (int)sh.dtype);
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > kMaxM || g.ny > kMaxM || g.nz > kMaxNz)
        return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "voxel grid %dx%dx%d outside 1..%d x 1..%d x 1..%d", g.nx, g.ny,
                    g.nz, kMaxM, kMaxM, kMaxNz);
    if (!(g.dx > 0) || !(g.dy > 0) || !(g.dz > 0) || !std::isfinite(g.x0) || !std::isfinite(g.y0) ||
        !std::isfinite(g.z0) || !std::isfinite(g.dx) || !std::isfinite(g.dy) || !std::isfinite(g.dz))
        return fail(MMSAR_ERR_INVALID_ARG, "grid pitches must be finite and > 0");
    if (o.compensate < 0 || o.compensate > 2) return fail(MMSAR_ERR_INVALID_ARG, "compensate must be 0, 1 or 2");
    p.mx = o.mx > 0 ? o.mx : next_pow2(g.nx);
    p.my = o.my > 0 ? o.my : next_pow2(g.ny);
    if (p.mx < 16) p.mx = 16;
    if (p.my < 16) p.my = 16;
    if (!is_pow2(p.mx) || !is_pow2(p.my) || p.mx > kMaxM || p.my > kMaxM || p.mx < g.nx || p.my < g.ny)
        return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "spectral grid %dx%d must be powers of two in 16..%d covering %dx%d",
                    p.mx, p.my, kMaxM, g.nx, g.ny);
    const double tol = o.nufft_tol > 0 ? o.nufft_tol : 1e-3;
    if (!(tol < 1.0)) return fail(MMSAR_ERR_INVALID_ARG, "nufft_tol must be < 1");
    p.w = width_for_tol(tol);
    p.mrx = 2 * p.mx;
    p.mry = 2 * p.my;
    p.mrz = next_pow2(2 * g.nz);
    if (p.mrz < 32) p.mrz = 32;
    p.n_kc = (sh.n_k + kKC - 1) / kKC;
    p.nkp = p.n_kc * kKC;
    p.L = (int64_t)sh.n_tx * sh.n_rx * sh.n_pos;
    if (p.L > (int64_t)0x7fffffff / 2) return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "too many samples (%lld)", (long long)p.L);
    if (p.L * (int64_t)(2 * p.w + 7) >= ((int64_t)1 << 31) || p.L * kKC >= ((int64_t)1 << 31))
        return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "too many samples for 32-bit record indices (%lld)", (long long)p.L);
    p.nbx = p.mrx / kBin;
    p.nby = p.mry / kBin;
    p.n_bins = (int64_t)p.nbx * p.nby;
    p.spread_nf = 2;
    p.spread_warps = 4;   // the autotuner's choice on the realistic, large and most batched scans
    p.grouped = false;
    p.tc = 5;             // warp-specialised tensor-core gridding (0: FP32 FMA; all are autotuner options)
    p.wait_test = 0;
    p.G = p.L;
    p.zref_given = std::isfinite(o.z_ref);
    p.z_ref = p.zref_given ? o.z_ref : 0.0;
    p.z_scene = std::isfinite(o.z_scene) ? o.z_scene : g.z0 + 0.5 * (g.nz - 1) * g.dz;
    if (p.zref_given && o.compensate && !(p.z_scene > p.z_ref))
        return fail(MMSAR_ERR_INVALID_ARG, "z_scene (%g) must lie beyond z_ref (%g) on +z", p.z_scene, p.z_ref);
    // Greengard-Lee: tau = pi (w/2) / (M^2 sigma (sigma - 1/2)), sigma = 2
    p.tau_x = kPi * (0.5 * p.w) / ((double)p.mx * p.mx * 3.0);
    p.tau_y = kPi * (0.5 * p.w) / ((double)p.my * p.my * 3.0);
    const double mz = p.mrz / 2;
    p.tau_z = kPi * (0.5 * p.w) / (mz * mz * 3.0);
    // workspace layout
    size_t off = align256(sizeof(WsHeader));
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const size_t L = (size_t)p.L;
    p.off_partials = take(sizeof(double) * 128);
    p.off_aref = take(sizeof(int) * 64);   // before the bin counts: cleared with the header
    p.off_counts = take(sizeof(int) * (size_t)p.n_bins);
    p.off_offsets = take(sizeof(int) * ((size_t)p.n_bins + 1));
    p.off_cursor = take(sizeof(int) * (size_t)p.n_bins);
    p.off_binid = take(sizeof(int) * L);
    p.off_rec = take(sizeof(SampleRec) * L);
    p.off_phase = take(sizeof(uint2) * L);
    p.off_perm = take(sizeof(int) * L);
    p.off_dd = take(sizeof(int2) * L);
    p.off_wq = take(sizeof(float4) * (size_t)(2 * p.w + 7) * L);
    const size_t TR = (size_t)sh.n_tx * sh.n_rx;
    p.off_cls = take(sizeof(int) * (3 * TR + 1));
    p.off_grec = take(sizeof(GroupRec) * (size_t)p.G);
    p.off_gdd = take(sizeof(int2) * (size_t)p.G);
    p.off_gxq = take(sizeof(float4) * (size_t)(p.w + 3) * (size_t)p.G);
    p.off_goff = take(2 * sizeof(int4) * (size_t)p.G);
    p.off_yq = take(sizeof(float4) * (size_t)(p.w + 4) * L);
    p.off_trec = take(sizeof(int4) * L);
    p.off_sexp = take((size_t)((p.n_kc + 1) / 2) * L);
    p.off_shat = take(sizeof(float2) * (size_t)((p.n_kc + 1) / 2) * L * 2 * kKC);   // 64-frequency groups
    const size_t G = sizeof(float2) * (size_t)p.n_kc * p.mry * p.mrx * kKC;
    const size_t S = sizeof(float2) * (size_t)p.mx * p.my * p.nkp;
    const size_t B = sizeof(float2) * (size_t)p.mx * g.ny * g.nz;
    const size_t A = sizeof(float2) * (size_t)p.n_kc * p.mry * p.mx * kKC;
    const size_t Z = sizeof(float2) * (size_t)p.mx * p.my * g.nz;
    // G -> (FFT x') -> A -> (FFT y') -> S [in G's region] -> (Stolt) -> Z [in A's region]
    //   -> (IFFT k_y) -> B [in G's region] -> (IFFT k_x) -> vol
    p.off_G = take(std::max(G, std::max(S, B)));
    p.off_S = p.off_G;
    p.off_B = p.off_G;
    p.off_A = take(std::max(A, Z));
    p.off_Z = p.off_A;
    p.ws_bytes = off;
    return MMSAR_OK;
}

}  // namespace mmsar

using namespace mmsar;

extern "C" {

void mmsar_options_default(mmsar_options *opt) {
    if (!opt) return;
    opt->z_ref = NAN;
    opt->z_scene = NAN;
    opt->compensate = 1;
    opt->nufft_tol = 1e-3;
    opt->mx = 0;
    opt->my = 0;
}

mmsar_status mmsar_plan_create(mmsar_plan **out, const mmsar_shape *shape, const mmsar_grid *grid,
                               const mmsar_options *opt) {
    if (!out || !shape || !grid) return fail(MMSAR_ERR_INVALID_ARG, "null argument to mmsar_plan_create");
    *out = nullptr;
    mmsar_options o;
    if (opt)
        o = *opt;
    else
        mmsar_options_default(&o);
    mmsar_plan *pl = new (std::nothrow) mmsar_plan();
    if (!pl) return fail(MMSAR_ERR_OUT_OF_MEMORY, "host allocation of the plan failed");
    const mmsar_status st = build_plan(pl->p, *shape, *grid, o);
    if (st != MMSAR_OK) {
        delete pl;
        return st;
    }
    *out = pl;
    return MMSAR_OK;
}

mmsar_status mmsar_plan_workspace_bytes(const mmsar_plan *plan, size_t *bytes) {
    if (!plan || !bytes) return fail(MMSAR_ERR_INVALID_ARG, "null argument to mmsar_plan_workspace_bytes");
    *bytes = plan->p.ws_bytes;
    return MMSAR_OK;
}

mmsar_status mmsar_plan_info(const mmsar_plan *plan, int *kernel_width, int *mx, int *my,
                             int *kernels_per_image) {
    if (!plan) return fail(MMSAR_ERR_INVALID_ARG, "null plan");
    if (kernel_width) *kernel_width = plan->p.w;
    if (mx) *mx = plan->p.mx;
    if (my) *my = plan->p.my;
    if (kernels_per_image) *kernels_per_image = plan->p.L > 0 ? kKernelsPerImage : 0;
    return MMSAR_OK;
}

mmsar_status mmsar_plan_set_tiles(mmsar_plan *plan, const mmsar_tiles *tiles) {
    if (!plan || !tiles) return fail(MMSAR_ERR_INVALID_ARG, "null plan or tiles");
    if (tiles->grid_freqs_per_lane != 1 && tiles->grid_freqs_per_lane != 2 && tiles->grid_freqs_per_lane != 4)
        return fail(MMSAR_ERR_INVALID_ARG, "grid_freqs_per_lane must be 1, 2 or 4");
    if (tiles->grid_warps_per_cta != 4 && tiles->grid_warps_per_cta != 8)
        return fail(MMSAR_ERR_INVALID_ARG, "grid_warps_per_cta must be 4 or 8");
    if (tiles->grid_grouped != 0 && tiles->grid_grouped != 1)
        return fail(MMSAR_ERR_INVALID_ARG, "grid_grouped must be 0 or 1");
    if (tiles->grid_grouped && tiles->grid_freqs_per_lane == 4)
        return fail(MMSAR_ERR_INVALID_ARG, "the grouped form takes 1 or 2 frequencies per lane");
    if (tiles->grid_grouped && (int64_t)plan->p.shape.n_tx * plan->p.shape.n_rx > kMaxPairsGrouped)
        return fail(MMSAR_ERR_UNSUPPORTED_SIZE, "grouped gridding takes at most %d Tx/Rx pairs", kMaxPairsGrouped);
    if (tiles->grid_tensor_cores < 0 || tiles->grid_tensor_cores > 5)
        return fail(MMSAR_ERR_INVALID_ARG, "grid_tensor_cores must be 0 .. 5");
    plan->p.spread_nf = tiles->grid_freqs_per_lane;
    plan->p.spread_warps = tiles->grid_warps_per_cta;
    plan->p.grouped = tiles->grid_grouped != 0;
    plan->p.tc = tiles->grid_tensor_cores;
    return MMSAR_OK;
}

mmsar_status mmsar_plan_set_wait_test(mmsar_plan *plan, int on) {
    if (!plan) return fail(MMSAR_ERR_INVALID_ARG, "null plan");
    if (on != 0 && on != 1) return fail(MMSAR_ERR_INVALID_ARG, "on must be 0 or 1");
    plan->p.wait_test = on;
    return MMSAR_OK;
}

mmsar_status mmsar_plan_get_tiles(const mmsar_plan *plan, mmsar_tiles *tiles) {
    if (!plan || !tiles) return fail(MMSAR_ERR_INVALID_ARG, "null plan or tiles");
    tiles->grid_freqs_per_lane = plan->p.spread_nf;
    tiles->grid_warps_per_cta = plan->p.spread_warps;
    tiles->grid_grouped = plan->p.grouped ? 1 : 0;
    tiles->grid_tensor_cores = plan->p.tc;
    return MMSAR_OK;
}

int mmsar_stage_count(void) { return kStages; }

const char *mmsar_stage_name(int stage) {
    static const char *names[kStages] = {"prep", "compensate", "grid", "fft_x", "fft_y", "stolt", "ifft_y", "ifft_x"};
    return (stage >= 0 && stage < kStages) ? names[stage] : "";
}

mmsar_status mmsar_plan_set_stage_events(mmsar_plan *plan, void *const *events, int n) {
    if (!plan) return fail(MMSAR_ERR_INVALID_ARG, "null plan");
    if (n == 0) {
        plan->p.n_events = 0;
        return MMSAR_OK;
    }
    if (!events || n != kStages + 1) return fail(MMSAR_ERR_INVALID_ARG, "need %d events", kStages + 1);
    for (int i = 0; i < n; ++i) plan->p.events[i] = reinterpret_cast<cudaEvent_t>(events[i]);
    plan->p.n_events = n;
    return MMSAR_OK;
}

// The argument checks of one image (shared by the single and batched calls).
static mmsar_status check_request(const mmsar_plan *plan, const void *workspace, size_t workspace_bytes,
                                  const void *echo, const float *echo_scale, const double *pos, const double *tx,
                                  const double *rx, const void *vol) {
    if (!plan) return fail(MMSAR_ERR_INVALID_ARG, "null plan");
    const Plan &p = plan->p;
    if (!workspace || !vol) return fail(MMSAR_ERR_INVALID_ARG, "null workspace or output volume");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(MMSAR_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < p.ws_bytes)
        return fail(MMSAR_ERR_OUT_OF_MEMORY, "workspace of %zu bytes is smaller than the %zu required",
                    workspace_bytes, p.ws_bytes);
    if (reinterpret_cast<uintptr_t>(vol) % 8 != 0) return fail(MMSAR_ERR_INVALID_ARG, "vol must be 8-byte aligned");
    if (p.L > 0 && (!echo || !pos || !tx || !rx)) return fail(MMSAR_ERR_INVALID_ARG, "null input pointer");
    if (p.L > 0 && p.shape.dtype != MMSAR_ECHO_C64 && !echo_scale)
        return fail(MMSAR_ERR_INVALID_ARG, "scaled FP16/BF16 echo needs echo_scale");
    return MMSAR_OK;
}

mmsar_status mmsar_image(mmsar_plan *plan, void *workspace, size_t workspace_bytes, const void *echo,
                         const float *echo_scale, const double *pos, const double *tx, const double *rx, void *vol,
                         void *stream) {
    const mmsar_status st = check_request(plan, workspace, workspace_bytes, echo, echo_scale, pos, tx, rx, vol);
    if (st != MMSAR_OK) return st;
    const Plan &p = plan->p;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t vol_bytes = sizeof(float2) * (size_t)p.grid.nx * p.grid.ny * p.grid.nz;
    cudaError_t e = cudaMemsetAsync(workspace, 0, p.off_counts + sizeof(int) * (size_t)p.n_bins, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the workspace header");
    if (p.L == 0) {
        e = cudaMemsetAsync(vol, 0, vol_bytes, s);
        return e == cudaSuccess ? MMSAR_OK : cuda_fail(e, "clearing the volume");
    }
#define MMSAR_STEP(call, what)                             \
    do {                                                   \
        cudaError_t ee = (call);                           \
        if (ee != cudaSuccess) return cuda_fail(ee, what); \
    } while (0)
#define MMSAR_MARK(i) \
    if (p.n_events) MMSAR_STEP(cudaEventRecord(p.events[i], s), "recording a stage event")
    MMSAR_MARK(0);
    MMSAR_STEP(launch_zref(p, workspace, pos, tx, rx, s), "z_ref");
    MMSAR_STEP(launch_geometry(p, workspace, pos, tx, rx, s), "geometry");
    MMSAR_STEP(launch_bin_scatter(p, workspace, s), "bin scatter");
    MMSAR_MARK(1);
    MMSAR_STEP(launch_compensate(p, workspace, echo, echo_scale, s), "compensation, bin sort and gridding weights");
    MMSAR_MARK(2);
    MMSAR_STEP(p.tc ? launch_grid_tc(p, workspace, s)
                    : (p.grouped ? launch_spread_groups(p, workspace, s) : launch_spread(p, workspace, s)),
               "gridding");
    MMSAR_MARK(3);
    MMSAR_STEP(launch_fft_x(p, workspace, s), "FT_2D along x'");
    MMSAR_MARK(4);
    MMSAR_STEP(launch_fft_y(p, workspace, s), "FT_2D along y'");
    MMSAR_MARK(5);
    MMSAR_STEP(launch_stolt(p, workspace, s), "Stolt");
    MMSAR_MARK(6);
    MMSAR_STEP(launch_ifft_y(p, workspace, s), "IFT along k_y");
    MMSAR_MARK(7);
    MMSAR_STEP(launch_ifft_x(p, workspace, vol, s), "IFT along k_x");
    MMSAR_MARK(8);
#undef MMSAR_MARK
#undef MMSAR_STEP
    return MMSAR_OK;
}

mmsar_status mmsar_image_batch(const mmsar_request *reqs, int n, void *const *streams, int n_streams) {
    if (n < 0 || (n > 0 && !reqs) || n_streams < 1 || !streams)
        return fail(MMSAR_ERR_INVALID_ARG, "bad arguments to mmsar_image_batch");
    for (int i = 0; i < n; ++i) {
        const mmsar_request &r = reqs[i];
        const mmsar_status st = mmsar_image(r.plan, r.workspace, r.workspace_bytes, r.echo, r.echo_scale, r.pos, r.tx,
                                            r.rx, r.vol, streams[i % n_streams]);
        if (st != MMSAR_OK) return st;
    }
    return MMSAR_OK;
}

mmsar_status mmsar_image_batch_fused(const mmsar_request *reqs, int n, void *stream, int *launches) {
    if (launches) *launches = 0;
    if (n < 0 || (n > 0 && !reqs)) return fail(MMSAR_ERR_INVALID_ARG, "bad arguments to mmsar_image_batch_fused");
    std::vector<mmsar_request> live;
    live.reserve((size_t)n);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n; ++i) {
        const mmsar_request &r = reqs[i];
        const mmsar_status st =
            check_request(r.plan, r.workspace, r.workspace_bytes, r.echo, r.echo_scale, r.pos, r.tx, r.rx, r.vol);
        if (st != MMSAR_OK) return st;
    }
    int count = 0;
    for (int i = 0; i < n; ++i) {
        const mmsar_request &r = reqs[i];
        const Plan &p = r.plan->p;
        if (p.L > 0) {
            live.push_back(r);
        } else {   // no samples: the volume is zero
            const size_t vol_bytes = sizeof(float2) * (size_t)p.grid.nx * p.grid.ny * p.grid.nz;
            const cudaError_t e = cudaMemsetAsync(r.vol, 0, vol_bytes, s);
            if (e != cudaSuccess) return cuda_fail(e, "clearing a volume");
            ++count;
        }
    }
    const int m = (int)live.size();
    if (m == 0) {
        if (launches) *launches = count;
        return MMSAR_OK;
    }
    const mmsar_request *r = live.data();
    g_fused_launches = 0;
#define MMSAR_STEP(call, what)                             \
    do {                                                   \
        cudaError_t ee = (call);                           \
        if (ee != cudaSuccess) return cuda_fail(ee, what); \
    } while (0)
    MMSAR_STEP(launch_clear_multi(r, m, s), "clearing the workspace headers");
    MMSAR_STEP(launch_zref_multi(r, m, s), "z_ref");
    MMSAR_STEP(launch_geometry_multi(r, m, s), "geometry");
    MMSAR_STEP(launch_bin_scatter_multi(r, m, s), "bin scatter");
    MMSAR_STEP(launch_compensate_multi(r, m, s), "compensation, bin sort and gridding weights");
    MMSAR_STEP(launch_spread_multi(r, m, s), "gridding");
    MMSAR_STEP(launch_grid_tc_multi(r, m, s), "gridding on the tensor cores");
    MMSAR_STEP(launch_fft_multi(r, m, 0, s), "FT_2D along x'");
    MMSAR_STEP(launch_fft_multi(r, m, 1, s), "FT_2D along y'");
    MMSAR_STEP(launch_stolt_multi(r, m, s), "Stolt");
    MMSAR_STEP(launch_fft_multi(r, m, 2, s), "IFT along k_y");
    MMSAR_STEP(launch_fft_multi(r, m, 3, s), "IFT along k_x");
#undef MMSAR_STEP
    if (launches) *launches = count + g_fused_launches;
    return MMSAR_OK;
}

mmsar_status mmsar_poll_error(const void *workspace, void *stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!workspace) {   // the built-in scratch area of mmsar_image_static on the current device
        void *ws = nullptr;
        const mmsar_status st = static_workspace_address(s, &ws);
        if (st != MMSAR_OK) return st;
        workspace = ws;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronising the stream");
    int word = 0;
    e = cudaMemcpy(&word, workspace, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the error word");
    if (word) {
        e = cudaMemset(const_cast<void *>(workspace), 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "clearing the error word");
    }
    if (word & kErrNonfinite) return fail(MMSAR_ERR_NONFINITE, "non-finite value in the echo or the geometry");
    if (word & kErrTimeout)
        return fail(MMSAR_ERR_DEVICE_TIMEOUT,
                    "a bounded device-side wait of the tensor-core gridding gave up: the image is void");
    if (word & kErrGeometry)
        return fail(MMSAR_ERR_INVALID_ARG, "z_scene does not lie beyond the reference plane z_ref (Z_c <= 0)");
    if (word) return fail(MMSAR_ERR_CUDA, "device error word 0x%x", word);
    return MMSAR_OK;
}

size_t mmsar_peak_scratch_bytes(int64_t n) { return peak_scratch_bytes(n); }

mmsar_status mmsar_peak(const void *vol, int64_t n, void *scratch, void *result, void *stream) {
    if (!vol || !scratch || !result || n < 1) return fail(MMSAR_ERR_INVALID_ARG, "bad argument to mmsar_peak");
    cudaError_t e = launch_peak(vol, n, scratch, result, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMSAR_OK : cuda_fail(e, "peak");
}

const char *mmsar_last_error(void) { return g_last_error.c_str(); }

void mmsar_plan_destroy(mmsar_plan *plan) { delete plan; }

const char *mmsar_version(void) { return "mmsar 0.1 (sm_103a)"; }

}  // extern "C"
