// Internal declarations shared by the translation units of libmmsar.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mmsar.h"

namespace mmsar {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kKC = 32;       // frequencies per k-chunk (one per lane)
constexpr int kBin = 4;       // spreading bin / warp block edge, in grid cells
constexpr int kMaxNk = 1024;
constexpr int kMaxM = 1024;   // spectral grid per axis (FFT length 2M <= 2048)
constexpr int kMaxNz = 256;

// Error bits of the device error word (one per mmsar_status code).
constexpr int kErrNonfinite = 1 << MMSAR_ERR_NONFINITE;
constexpr int kErrGeometry = 1 << MMSAR_ERR_INVALID_ARG;
constexpr int kErrTimeout = 1 << MMSAR_ERR_DEVICE_TIMEOUT;

// Device-visible header at offset 0 of the workspace.
struct WsHeader {
    int error;          // OR of kErr* bits
    int n_valid;        // samples that were binned
    double z_ref;       // resolved reference plane
    // first gridding cell of any sample, unwrapped (min / max over samples)
    int u_min, u_max, v_min, v_max;
    // occupied window of the periodic gridding grid: cells lo .. lo + len - 1
    // (mod the grid size) can be nonzero; everything else is known zero
    int u_lo, u_len, v_lo, v_len;
    int zref_done;      // blocks of the z_ref reduction that have finished
    int geom_done;      // blocks of the geometry pass that have finished
    double inv_4zc;     // 1 / (4 Z_c), Z_c = z_scene - z_ref (0 without compensation)
    double zc;          // Z_c (0 without compensation)
    // grouped gridding: x-offset classes of the Tx/Rx pairs, and the largest
    // span of first y cells inside one group
    int n_classes, vspan_max;
    double pad[6];
};
static_assert(sizeof(WsHeader) == 128, "header size");

// Per-group record of the grouped gridding path: the samples of one position
// whose Tx/Rx pairs have the same x offset share x' (Eq. 3) and so the x
// weights; they differ in y.
struct GroupRec {
    int u0;             // first x cell, wrapped into [0, Mr)
    int v0min;          // first y cell of the group's lowest element, wrapped
    float fx;           // x position minus u0, in cells
    int vspan;          // highest minus lowest first y cell of its elements
};

// Largest Tx x Rx pair count of the grouped gridding path: a group's member
// offsets (first y cell above the group's lowest, 16 bits each) fit one
// 32-byte record.
constexpr int kMaxPairsGrouped = 16;

// Per-sample gridding record (sorted by bin).
struct SampleRec {
    int u0, v0;         // first grid cell of the support, wrapped into [0, Mr)
    float fx, fy;       // exact grid position minus (u0, v0), in cells
};

// Everything the kernels need, resolved on the host (plain values).
struct Plan {
    mmsar_shape shape;
    mmsar_grid grid;
    mmsar_options opt;
    int w;              // Gaussian taps per axis
    int mx, my;         // spectral modes per axis
    int mrx, mry;       // oversampled gridding grid (2 mx, 2 my)
    int mrz;            // z gridding grid (power of two >= max(32, 2 nz))
    int n_kc;           // k chunks of 32
    int nkp;            // n_kc * 32
    int64_t L;          // n_tx n_rx n_pos
    int nbx, nby;       // bins per axis (mrx / 4, mry / 4)
    int spread_nf;      // gridding launch shape: frequencies per lane (1, 2 or 4)
    int spread_warps;   //   and warps per CTA (4: 8 x 8 cells, 8: 16 x 8 cells; half as tall for 4)
    bool grouped;       // gridding by groups of samples sharing x' (else per sample)
    int tc;             // gridding on the tensor cores, pipeline variant 1..5 (grid_tc.cu); 0: the FP32 forms above
    int wait_test;      // 1: the warp-specialised gridding's bounded-wait expiry is exercised (tests only)
    int64_t G;          // group slots: n_tx n_rx n_pos (every class may be a single pair)
    int64_t n_bins;
    bool zref_given;
    double z_ref;       // when given
    double z_scene;     // resolved (grid centre when NaN)
    double tau_x, tau_y, tau_z;
    // workspace layout (byte offsets)
    size_t off_counts, off_offsets, off_cursor, off_binid, off_rec, off_phase, off_perm;
    size_t off_dd, off_wq;   // per sorted sample: (in-bin cell offset, sample index); Gaussian weight quads
    size_t off_partials;     // per-block sums of the z_ref reduction
    size_t off_cls;          // pair classes [TR], class starts [TR + 1], members [TR]
    size_t off_grec;         // per group: GroupRec [G]
    size_t off_gdd, off_gxq; // per sorted group: (in-bin offsets, group index); x weight quads [w + 3]
    size_t off_goff;         // per sorted group: its members' y offsets, uint16 x 16
    size_t off_yq;           // per sample (original order): offset header + y weight quads [w + 4]
    size_t off_trec;         // tensor-core gridding: per sorted sample (index, first cell, fractions)
    size_t off_sexp;         // tensor-core gridding: per (64-frequency group, sample) normalisation exponent
    size_t off_aref;         // tensor-core gridding: per group max of 127 - exponent (cleared per image)
    size_t off_shat, off_G, off_A, off_S, off_Z, off_B;
    size_t ws_bytes;
    // optional per-stage timing events (caller-owned)
    int n_events;
    cudaEvent_t events[16];
};

constexpr int kStages = 8;
constexpr int kKernelsPerImage = 10;

}  // namespace mmsar

struct mmsar_plan {
    mmsar::Plan p;
};

namespace mmsar {

// ---------------------------------------------------------------- launchers
// All return cudaSuccess or the launch error.
cudaError_t launch_zref(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                        cudaStream_t s);
cudaError_t launch_geometry(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                            cudaStream_t s);
cudaError_t launch_bin_scatter(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_compensate(const Plan &p, void *ws, const void *echo, const float *scale, cudaStream_t s);
cudaError_t launch_spread(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_spread_groups(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_grid_tc(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_grid_tc_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_fft_x(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_fft_y(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_stolt(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_ifft_y(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_ifft_x(const Plan &p, void *ws, void *vol, cudaStream_t s);
cudaError_t launch_peak(const void *vol, int64_t n, void *scratch, void *result, cudaStream_t s);
size_t peak_scratch_bytes(int64_t n);

// ---------------------------------------------------------------- fused batches
// A fused launch runs one stage for up to kBatchMax scans that use the same
// kernel instance: the blocks of scan i are blocks start[i] .. start[i+1]-1
// of the launch, and the scans' arguments travel in one kernel parameter
// block (__grid_constant__, a few KB).
constexpr int kBatchMax = 32;

template <typename A>
struct BatchTable {
    A a[kBatchMax];
    int start[kBatchMax + 1];
    int n;
};

// The scan of this block of a fused launch (binary search over the block
// starts), the block's index inside that scan and the scan's block count.
template <typename A>
__device__ __forceinline__ int batch_scan(const BatchTable<A> &t, int &bid, int &nb) {
    const int b = blockIdx.x;
    int lo = 0, hi = t.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.start[mid] <= b) lo = mid; else hi = mid;
    }
    bid = b - t.start[lo];
    nb = t.start[lo + 1] - t.start[lo];
    return lo;
}

// Copy the block's scan arguments to shared memory once (every thread calls
// it; the copy is visible after it returns), so that the kernel body reads
// them with plain shared-memory loads.
template <typename A>
__device__ __forceinline__ void batch_args(const BatchTable<A> &t, int s, A *dst) {
    static_assert(sizeof(A) % 4 == 0, "argument block of whole words");
    const int *src = reinterpret_cast<const int *>(&t.a[s]);
    int *d = reinterpret_cast<int *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = src[i];
    __syncthreads();
}

// Host side: launch fn(key, table, blocks) once per group of scans with the
// same key (in order of first appearance), in chunks of kBatchMax.
// kernels the fused launches of the current batch call have made (host)
inline thread_local int g_fused_launches = 0;

template <typename A, typename K, typename F>
cudaError_t launch_groups(int n, const K *keys, const A *args, const int *blocks, F fn) {
    // kernel parameters may take up to 32 KB (CUDA 12.1+); stay well inside
    static_assert(sizeof(BatchTable<A>) <= 16384, "fused-launch argument table too large");
    std::vector<char> done((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        if (done[i] || blocks[i] <= 0) continue;
        BatchTable<A> t;
        t.n = 0;
        int total = 0;
        for (int j = i; j < n; ++j) {
            if (done[j] || blocks[j] <= 0 || !(keys[j] == keys[i])) continue;
            done[j] = 1;
            t.a[t.n] = args[j];
            t.start[t.n] = total;
            total += blocks[j];
            ++t.n;
            if (t.n == kBatchMax) {
                t.start[t.n] = total;
                const cudaError_t e = fn(keys[i], t, total);
                if (e != cudaSuccess) return e;
                ++g_fused_launches;
                t.n = 0;
                total = 0;
            }
        }
        if (t.n > 0) {
            t.start[t.n] = total;
            const cudaError_t e = fn(keys[i], t, total);
            if (e != cudaSuccess) return e;
            ++g_fused_launches;
        }
    }
    return cudaSuccess;
}

// Fused launches of the stages of mmsar_image for n requests (same order and
// meaning as the single-scan launchers; requests without samples excluded).
cudaError_t launch_clear_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_zref_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_geometry_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_bin_scatter_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_compensate_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_spread_multi(const mmsar_request *r, int n, cudaStream_t s);
cudaError_t launch_fft_multi(const mmsar_request *r, int n, int stage, cudaStream_t s);   // stage 0..3: x, y, iy, ix
cudaError_t launch_stolt_multi(const mmsar_request *r, int n, cudaStream_t s);

// Record a formatted message for mmsar_last_error() and return `st`.
mmsar_status report_error(mmsar_status st, const char *fmt, ...);

// Device address of the built-in scratch area of mmsar_image_static on the
// current device (looked up afresh unless `s` is being captured).
mmsar_status static_workspace_address(cudaStream_t s, void **out);

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute is per device; the first launch on each device sets it).
cudaError_t ensure_smem_attr(const void *func, size_t bytes);

// Column-batched FFT along the row axis of a strided 2-D tile set (see
// fft_kernels.cu).  Row r of a tile is placed at FFT index (r + in_shift) mod L;
// output row o takes FFT index (o - n_out/2) mod L and is scaled by
//   scale * (gauss_tau > 0 ? exp(f^2 * gauss_tau) : 1),  f = o - n_out/2.
struct ColumnFFT {
    int L;              // FFT length (power of two, 16..2048)
    int sign;           // -1 forward, +1 inverse (unnormalised)
    const float2 *in;
    float2 *out;
    int n_in;           // rows read (<= L)
    int in_shift;
    long long in_row, in_t1, in_t2;     // element strides
    int n_out;          // rows written (<= L)
    long long out_row, out_t1, out_t2;
    int ncols;          // contiguous columns per tile
    int nt1, nt2;       // tile counts
    // optional device windows (lo, len), periodic: input rows outside
    // in_win (period n_in) are taken as zero without being read; tiles t2
    // outside tile_win (period nt2) are skipped entirely (nothing written)
    const int *in_win;
    const int *tile_win;
    float scale;
    float gauss_tau;
};
cudaError_t launch_column_fft(const ColumnFFT &a, cudaStream_t s);

}  // namespace mmsar
