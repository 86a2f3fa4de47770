// k_z filter and Stolt step of Eq. 15-16 for every spectral column (k_x, k_y).
//
// For column (m, n) and frequency sample k (Eq. 14, Eq. 15 with P(f) = 1):
//     k_z = sqrt(4 k^2 - k_x^2 - k_y^2)        (dropped when not positive)
//     c_k = S(m, n, k) * k_z * exp(+j k_z (z_c - z_ref)),   z_c = z0 + (nz/2) dz
// and the image column over depth is the sum over the non-uniform k_z samples
//     Z(m, n, q) = sum_k c_k exp(+j q' t_k),   t_k = k_z dz,  q' = q - nz/2,
// i.e. exp(+j k_z (z_q - z_ref)) split at the centre slice.  The sum is the
// Stolt interpolation S plus the inverse transform over k_z of Eq. 16, done
// as a 1-D fast Gaussian gridding NUFFT (Sec. III): every k_z sample is
// spread onto an oversampled periodic grid of MRZ points, the grid is
// transformed by an inverse FFT and the Gaussian is deconvolved.
//
// One warp per column, or per pair of mirror columns (+-k_x, k_y), which
// share every k_z sample position, phase factor and weight.  Because k_z grows with k, the samples of a column are already
// sorted along the gridding axis: each lane spreads a contiguous run of them
// into a small window of grid points kept in registers (one window per column
// of the pair), and the windows are then summed per grid point in lane order
// -- no atomics, a fixed summation order.  The FFT then runs over the columns
// of the CTA in shared memory (fft.cuh).
#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

struct StoltArgs {
    const float2 *S;        // [mx][my][nkp]
    float2 *Z;              // [mx][my][nz]
    const WsHeader *hdr;
    int mx, my, nk, nkp, nz, w;
    float kx_step, ky_step;    // 2 pi / (M d)
    float k0_hi, k0_lo, dk;    // 2 pi f0 / c as a float pair, 2 pi df / c
    float cells_per_kz;        // dz MRZ / (2 pi)
    double z_c;                // z0 + (nz / 2) dz
    float kappa;
    float deapod_scale;        // sqrt(pi / tau_z) / MRZ
    float tau_z;
};

constexpr int kStoltCols = 8;

// complex elements of a warp's scratch region (even, so every region starts
// on 16 bytes): the larger of the lanes' windows of WP points for NC
// columns and the fallback's staged samples of one column (nk values + nk
// floats)
__host__ __device__ inline int stolt_warp_scratch(int nk, int WP, int NC) {
    const int a = NC * 32 * WP, b = nk + (nk + 1) / 2;
    const int m = a > b ? a : b;
    return (m + 1) & ~1;
}

// NC = 1: warp w of block b takes spectral column 8 b + w.  NC = 2: it takes
// the mirror pair (k_x, k_y), (-k_x, k_y) -- pair (cx, n), cx <= Mx/2, one or
// two columns (index 0 and Mx/2 have no mirror on the grid).  The columns of
// a pair share k_x^2 + k_y^2 and hence every k_z sample position, phase
// factor and Gaussian weight (computed once, bit for bit as for a single
// column); only the spectrum values differ.  GP: row pitch of the grid tile
// of 8 NC columns.
template <int MRZ, int WR, int GP, int NC>
__device__ __forceinline__ void stolt_body(const StoltArgs &a, int bid) {
    extern __shared__ float2 smem[];
    constexpr int WP = WR + 1;                            // padded pitch of a lane's window
    float2 *grid = smem;                                  // [MRZ][GP], column warp * NC + ci
    float2 *tw = grid + MRZ * GP;                         // [MRZ]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // per-warp scratch: either the lanes' register windows [NC][32][WP] or, on
    // the fallback path, one column's staged samples (values [nk], grid positions [nk])
    const int wscr = stolt_warp_scratch(a.nk, WP, NC);
    float2 *scratch = tw + MRZ + warp * wscr;
    int *jlo_s = reinterpret_cast<int *>(tw + MRZ + kStoltCols * wscr);   // [8 * 32]
    __shared__ float turns_per_kz_s;   // (z_c - z_ref) / (2 pi): once per CTA (z_ref lives on the device)
    if (tid == 0) turns_per_kz_s = (float)((a.z_c - a.hdr->z_ref) * (0.5 / kPi));
    // the warp's columns (-1: none) and their shared (k_x, k_y) magnitudes
    int cols[NC];
    int om, on;
    bool live;
    if constexpr (NC == 1) {
        const int col = bid * kStoltCols + warp;
        live = col < a.mx * a.my;
        om = col / a.my;
        on = col - om * a.my;
        cols[0] = live ? col : -1;
    } else {
        static_assert(NC == 2, "one column or a mirror pair per warp");
        const int cls = bid * kStoltCols + warp;
        live = cls < (a.mx / 2 + 1) * a.my;
        om = cls / a.my;
        on = cls - om * a.my;
        const bool px = om > 0 && om < a.mx / 2;
        cols[0] = live ? om * a.my + on : -1;
        cols[1] = live && px ? (a.mx - om) * a.my + on : -1;
    }
    for (int e = tid; e < MRZ * GP; e += 256) grid[e] = make_float2(0.f, 0.f);
    fill_twiddles<MRZ, +1>(tw, tid, 256);
    __syncthreads();
    if (live) {
        const float kx = (float)(om - a.mx / 2) * a.kx_step;
        const float ky = (float)(on - a.my / 2) * a.ky_step;
        const float kr2 = kx * kx + ky * ky;
        const float turns_per_kz = turns_per_kz_s;
        const float cells_per_kz = a.cells_per_kz;
        const float2 *Sc[NC];
#pragma unroll
        for (int ci = 0; ci < NC; ++ci) Sc[ci] = a.S + (long long)(cols[ci] < 0 ? 0 : cols[ci]) * a.nkp;
        const float hw = 0.5f * a.w;
        // k = 2 pi f / c on the uniform grid, formed as k0_hi + (k0_lo + k dk)
        // (k0 split into two floats): within half an ulp of the FP64 value
        const float k0_hi = a.k0_hi, k0_lo = a.k0_lo, dkf = a.dk;
        auto wavenumber = [&](int k) { return k0_hi + fmaf((float)k, dkf, k0_lo); };
        // k_z grows with k: the evanescent samples (4k^2 <= k_x^2 + k_y^2) form a prefix
        int kf = 0;
        for (int k0 = 0; k0 < a.nk; k0 += 32) {
            const int k = k0 + lane;
            float kv = 0.f;
            if (k < a.nk) kv = wavenumber(k);
            const bool evan = k < a.nk && 4.f * kv * kv - kr2 <= 0.f;
            kf += __popc(__ballot_sync(0xffffffffu, evan));
        }
        // Eq. 14-15 for one sample: grid position t (cells), k_z and the phase
        // factor exp(+j k_z (z_c - z_ref)); the weighted value of column ci is
        // then c = S(k) k_z (cs, sn)
        auto geometry = [&](int k, float &t, float &kz, float &cs, float &sn) {
            const float kv = wavenumber(k);
            kz = sqrtf(4.f * kv * kv - kr2);
            t = kz * cells_per_kz;
            float ph = kz * turns_per_kz;
            ph -= rintf(ph);                        // [-1/2, 1/2] turn
            __sincosf(6.283185307179586f * ph, &sn, &cs);
        };
        auto value = [&](int ci, int k, float kz, float cs, float sn) {
            const float2 sv = __ldg(Sc[ci] + k);
            return cmul(make_float2(sv.x * kz, sv.y * kz), make_float2(cs, sn));
        };
        if (kf < a.nk) {
            // Each lane spreads a contiguous run of samples (sorted along the
            // gridding axis) into a window of WR grid points held in registers;
            // the Gaussian weights of consecutive points follow the recurrence
            // w_{i+1} = w_i r_i, r_{i+1} = r_i exp(-2 kappa).
            const int nv = a.nk - kf;
            // grid position of sample k (as geometry() computes it)
            auto grid_pos = [&](int k) {
                const float kv = wavenumber(k);
                return sqrtf(4.f * kv * kv - kr2) * cells_per_kz;
            };
            // runs of equal sample counts; lanes past the last run are idle
            const int per = (nv + 31) / 32;
            int k_beg = kf + lane * per, k_end = min(a.nk, k_beg + per);
            int nact = (nv + per - 1) / per;
            int jl = 0x7fffffff;
            bool fits = true;
            if (k_beg < k_end) {
                jl = (int)ceilf(grid_pos(k_beg) - hw);
                fits = (int)ceilf(grid_pos(k_end - 1) - hw) + a.w - 1 - jl + 1 <= WR;
            }
            if (!__all_sync(0xffffffffu, fits)) {
                // near the evanescent edge k_z rises steeply and equal counts
                // span unequal depths: split the depth range into 32 equal
                // spans instead, lane l taking the samples with grid position
                // in [t_lo + l D, t_lo + (l + 1) D).  A boundary is the first
                // sample at or past its target, found from the closed-form
                // inverse of the k -> k_z map and corrected against grid_pos
                // itself, so neighbouring lanes agree on it exactly.
                const float t_lo = grid_pos(kf), D = (grid_pos(a.nk - 1) - t_lo) * (1.0f / 32.0f);
                auto first_at = [&](int m) {
                    if (m <= 0) return kf;
                    if (m >= 32) return a.nk;
                    const float target = fmaf((float)m, D, t_lo);
                    const float kz = target / cells_per_kz;
                    int k = (int)ceilf((0.5f * sqrtf(kz * kz + kr2) - k0_hi - k0_lo) / dkf);
                    k = min(max(k, kf), a.nk);
                    while (k > kf && grid_pos(k - 1) >= target) --k;
                    while (k < a.nk && grid_pos(k) < target) ++k;
                    return k;
                };
                k_beg = first_at(lane);
                k_end = first_at(lane + 1);
                nact = 32;
                // an empty run keeps a window start in order with its neighbours
                const float t_beg = k_beg < k_end ? grid_pos(k_beg) : fmaf((float)lane, D, t_lo);
                jl = (int)ceilf(t_beg - hw);
                fits = k_beg >= k_end || (int)ceilf(grid_pos(k_end - 1) - hw) + a.w - 1 - jl + 1 <= WR;
            }
            if (__all_sync(0xffffffffu, fits)) {
                float2 acc[NC][WR];
#pragma unroll
                for (int ci = 0; ci < NC; ++ci)
#pragma unroll
                    for (int i = 0; i < WR; ++i) acc[ci][i] = make_float2(0.f, 0.f);
                const float qk = __expf(-2.f * a.kappa);
                for (int k = k_beg; k < k_end; ++k) {
                    float t, kz, cs, sn;
                    geometry(k, t, kz, cs, sn);
                    const float d0 = t - (float)jl;
                    float wgt = __expf(-a.kappa * d0 * d0);
                    float rho = __expf(a.kappa * (2.f * d0 - 1.f));
                    // weights and ratios advance together: (w, r) *= (r, q)
                    float wv[WR];
                    float2 wr = make_float2(wgt, rho);
#pragma unroll
                    for (int i = 0; i < WR; ++i) {
                        wv[i] = wr.x;
                        wr = fmul2(wr, make_float2(wr.y, qk));
                    }
#pragma unroll
                    for (int ci = 0; ci < NC; ++ci) {
                        if (cols[ci] < 0) continue;
                        const float2 c = value(ci, k, kz, cs, sn);
#pragma unroll
                        for (int i = 0; i < WR; ++i) acc[ci][i] = ffma2(make_float2(wv[i], wv[i]), c, acc[ci][i]);
                    }
                }
#pragma unroll
                for (int ci = 0; ci < NC; ++ci) {
                    float2 *mine = scratch + (ci * 32 + lane) * WP;
#pragma unroll
                    for (int i = 0; i < WR; ++i) mine[i] = acc[ci][i];
                }
                jlo_s[warp * 32 + lane] = jl;
                __syncwarp();
                // sum the windows per grid point, lanes in a fixed order
                const int *jw = jlo_s + warp * 32;
                const int J_lo = jw[0], J_hi = jw[nact - 1] + WR - 1;
                for (int jb = J_lo; jb <= J_hi; jb += 32) {
                    const int j = jb + lane;
                    if (j <= J_hi) {
                        // windows start in non-decreasing order: the ones that
                        // reach point j start in [j - WR + 1, j], a run of lanes
                        // from the first start >= j - WR + 1 (binary search)
                        int lo = 0, hi = nact;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (jw[mid] < j - WR + 1) lo = mid + 1; else hi = mid;
                        }
#pragma unroll
                        for (int ci = 0; ci < NC; ++ci) {
                            if (cols[ci] < 0) continue;
                            const float2 *wb = scratch + ci * 32 * WP;
                            float2 sum = make_float2(0.f, 0.f);
                            for (int l2 = lo; l2 < nact; ++l2) {
                                const int o = j - jw[l2];
                                if (o < 0) break;
                                sum = cadd(sum, wb[l2 * WP + o]);
                            }
                            float2 &gref = grid[(j & (MRZ - 1)) * GP + warp * NC + ci];
                            gref = cadd(gref, sum);
                        }
                    }
                    __syncwarp();
                }
            } else {
                // a run that spans more than the register window (very coarse
                // depth sampling): stage one column's samples at a time and
                // gather each grid point from the samples in reach, found by
                // binary search
                float2 *cw = scratch;
                float *tw_ = reinterpret_cast<float *>(scratch + a.nk);
                for (int k = kf + lane; k < a.nk; k += 32) {
                    float t, kz, cs, sn;
                    geometry(k, t, kz, cs, sn);
                    tw_[k] = t;
                }
                __syncwarp();
                const int jlo = (int)ceilf(tw_[kf] - hw);
                const int jhi = (int)ceilf(tw_[a.nk - 1] - hw) + a.w - 1;
#pragma unroll
                for (int ci = 0; ci < NC; ++ci) {
                    if (cols[ci] < 0) continue;
                    for (int k = kf + lane; k < a.nk; k += 32) {
                        float t, kz, cs, sn;
                        geometry(k, t, kz, cs, sn);
                        cw[k] = value(ci, k, kz, cs, sn);
                    }
                    __syncwarp();
                    for (int jb = jlo; jb <= jhi; jb += 32) {
                        const int j = jb + lane;
                        if (j <= jhi) {
                            const float lo_t = (float)j - hw, hi_t = (float)j + hw;
                            int lo = kf, hi = a.nk;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (tw_[mid] > lo_t) hi = mid; else lo = mid + 1;
                            }
                            float2 acc = make_float2(0.f, 0.f);
                            for (int k = lo; k < a.nk && tw_[k] <= hi_t; ++k) {
                                const float d = tw_[k] - (float)j;
                                const float wgt = __expf(-a.kappa * d * d);
                                acc.x = fmaf(wgt, cw[k].x, acc.x);
                                acc.y = fmaf(wgt, cw[k].y, acc.y);
                            }
                            float2 &gref = grid[(j & (MRZ - 1)) * GP + warp * NC + ci];
                            gref = cadd(gref, acc);
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncthreads();
    smem_fft<MRZ, kStoltCols * NC, 256, +1, GP>(grid, tw);
#pragma unroll
    for (int ci = 0; ci < NC; ++ci) {
        if (cols[ci] < 0) continue;
        float2 *Zc = a.Z + (long long)cols[ci] * a.nz;
        for (int q = lane; q < a.nz; q += 32) {
            const int qp = q - a.nz / 2;
            const float sc = a.deapod_scale * __expf((float)(qp * qp) * a.tau_z);
            const float2 v = grid[(qp & (MRZ - 1)) * GP + warp * NC + ci];
            Zc[q] = make_float2(v.x * sc, v.y * sc);
        }
    }
}

// NC = 2 takes three CTAs per SM (the register bound); NC = 1 as many as fit
template <int MRZ, int WR, int GP, int NC>
__global__ void __launch_bounds__(256, NC == 2 ? 3 : 1) stolt_kernel(const StoltArgs a) {
    stolt_body<MRZ, WR, GP, NC>(a, blockIdx.x);
}

template <int MRZ, int WR, int GP, int NC>
__global__ void __launch_bounds__(256, NC == 2 ? 3 : 1)
    stolt_multi(const __grid_constant__ BatchTable<StoltArgs> t) {
    __shared__ StoltArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    stolt_body<MRZ, WR, GP, NC>(sa, bid);
}

// grid tile pitch: 8 NC columns plus one (consecutive grid points of one
// column then fall on different banks)
__host__ __device__ constexpr int stolt_pitch(int NC) { return kStoltCols * NC + 1; }

static size_t stolt_smem(int MRZ, int WR, int NC, int nk) {
    return (size_t)(MRZ * stolt_pitch(NC) + MRZ + kStoltCols * stolt_warp_scratch(nk, WR + 1, NC)) * sizeof(float2) +
           (size_t)kStoltCols * 32 * sizeof(int);
}

// mirror pairs for the 8-point window (w <= 6; two windows of more points
// no longer fit the registers) when three CTAs also fit in shared memory
static int stolt_nc(int MRZ, int WR, int nk) {
    return WR == 8 && MRZ <= 256 && stolt_smem(MRZ, WR, 2, nk) <= 75 * 1024 ? 2 : 1;
}

static int stolt_blocks(const StoltArgs &a, int nc) {
    const int units = nc == 2 ? (a.mx / 2 + 1) * a.my : a.mx * a.my;
    return (units + kStoltCols - 1) / kStoltCols;
}

// one scan (a) or a fused batch (t, the largest Nk of the batch sizing the scratch)
template <int MRZ, int WR, int NC>
static cudaError_t launch_mrz_wr_nc(const StoltArgs *a, const BatchTable<StoltArgs> *t, int blocks, cudaStream_t s) {
    constexpr int GP = stolt_pitch(NC);
    int nk = 0;
    if (a) {
        nk = a->nk;
    } else {
        for (int i = 0; i < t->n; ++i) nk = std::max(nk, t->a[i].nk);
    }
    const size_t smem = stolt_smem(MRZ, WR, NC, nk);
    if (a) {
        cudaError_t e = ensure_smem_attr((const void *)stolt_kernel<MRZ, WR, GP, NC>, smem);
        if (e != cudaSuccess) return e;
        stolt_kernel<MRZ, WR, GP, NC><<<stolt_blocks(*a, NC), 256, smem, s>>>(*a);
    } else {
        cudaError_t e = ensure_smem_attr((const void *)stolt_multi<MRZ, WR, GP, NC>, smem);
        if (e != cudaSuccess) return e;
        stolt_multi<MRZ, WR, GP, NC><<<blocks, 256, smem, s>>>(*t);
    }
    return cudaGetLastError();
}

template <int MRZ, int WR>
static cudaError_t launch_mrz_wr(int nc, const StoltArgs *a, const BatchTable<StoltArgs> *t, int blocks,
                                 cudaStream_t s) {
    if constexpr (WR == 8 && MRZ <= 256)   // (a 512-point tile of mirror pairs exceeds the budget)
        if (nc == 2) return launch_mrz_wr_nc<MRZ, WR, 2>(a, t, blocks, s);
    return launch_mrz_wr_nc<MRZ, WR, 1>(a, t, blocks, s);
}

// register window: w + 2 grid points rounded up to an even count
static int stolt_wr(int w) { return w <= 6 ? 8 : (w <= 8 ? 10 : (w <= 10 ? 12 : 14)); }

template <int MRZ>
static cudaError_t launch_mrz(int wr, int nc, const StoltArgs *a, const BatchTable<StoltArgs> *t, int blocks,
                              cudaStream_t s) {
    switch (wr) {
        case 8: return launch_mrz_wr<MRZ, 8>(nc, a, t, blocks, s);
        case 10: return launch_mrz_wr<MRZ, 10>(nc, a, t, blocks, s);
        case 12: return launch_mrz_wr<MRZ, 12>(nc, a, t, blocks, s);
        default: return launch_mrz_wr<MRZ, 14>(nc, a, t, blocks, s);
    }
}

// key: MRZ << 8 | register window << 2 | mirror pairs
static int stolt_key_nc(int key) { return (key & 1) ? 2 : 1; }

static cudaError_t stolt_dispatch(int key, const StoltArgs *a, const BatchTable<StoltArgs> *t, int blocks,
                                  cudaStream_t s) {
    const int wr = (key >> 2) & 63, nc = stolt_key_nc(key);
    switch (key >> 8) {
        case 32: return launch_mrz<32>(wr, nc, a, t, blocks, s);
        case 64: return launch_mrz<64>(wr, nc, a, t, blocks, s);
        case 128: return launch_mrz<128>(wr, nc, a, t, blocks, s);
        case 256: return launch_mrz<256>(wr, nc, a, t, blocks, s);
        case 512: return launch_mrz<512>(wr, nc, a, t, blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

static int stolt_describe(const Plan &p, void *ws, StoltArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.S = reinterpret_cast<const float2 *>(w + p.off_S);
    a.Z = reinterpret_cast<float2 *>(w + p.off_Z);
    a.hdr = reinterpret_cast<const WsHeader *>(w);
    a.mx = p.mx;
    a.my = p.my;
    a.nk = p.shape.n_k;
    a.nkp = p.nkp;
    a.nz = p.grid.nz;
    a.w = p.w;
    a.kx_step = (float)(2.0 * kPi / (p.mx * p.grid.dx));
    a.ky_step = (float)(2.0 * kPi / (p.my * p.grid.dy));
    const double k0 = 2.0 * kPi * p.shape.f0_hz / kC0;
    a.k0_hi = (float)k0;
    a.k0_lo = (float)(k0 - (double)a.k0_hi);
    a.dk = (float)(2.0 * kPi * p.shape.df_hz / kC0);
    a.cells_per_kz = (float)(p.grid.dz * p.mrz / (2.0 * kPi));
    a.z_c = p.grid.z0 + (p.grid.nz / 2) * p.grid.dz;
    a.kappa = (float)(1.5 * kPi / p.w);
    a.deapod_scale = (float)(std::sqrt(kPi / p.tau_z) / p.mrz);
    a.tau_z = (float)p.tau_z;
    const int wr = stolt_wr(p.w);
    return (p.mrz << 8) | (wr << 2) | (stolt_nc(p.mrz, wr, a.nk) / 2);
}

cudaError_t launch_stolt(const Plan &p, void *ws, cudaStream_t s) {
    StoltArgs a;
    const int key = stolt_describe(p, ws, a);
    return stolt_dispatch(key, &a, nullptr, 0, s);
}

cudaError_t launch_stolt_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<StoltArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n);
    for (int i = 0; i < n; ++i) {
        keys[i] = stolt_describe(r[i].plan->p, r[i].workspace, args[i]);
        blocks[i] = stolt_blocks(args[i], stolt_key_nc(keys[i]));
    }
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int key, const BatchTable<StoltArgs> &t, int total) {
                             return stolt_dispatch(key, nullptr, &t, total, s);
                         });
}

}  // namespace mmsar
