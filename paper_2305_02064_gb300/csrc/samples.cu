// Per-sample stage: reference plane, virtual-element geometry, binning and
// the phase compensation of Sec. II-C.
//
//  zref_kernel      z_ref = mean of z_l over all samples (when not given).
//  geometry_kernel  Eq. 3-4 virtual element (x', y'), separations d^x, d^y,
//                   d^z = z_l - z_ref; the residual beta of Eq. 12; the
//                   gridding position on the 2M-point oversampled aperture
//                   grid; the compensation phase as 32-bit fixed-point turns.
//  bin_*            counting sort of the samples by 4x4-cell bin.
//  compensate       Eq. 11, s_hat = s exp(+j k beta) in original sample
//                   order; the same launch finishes the binning (in-bin
//                   sort, gridding weight records).
//
// Precision: FP64 is used once per sample (geometry and the phase argument
// f0 beta / c, df beta / c reduced to [0, 1) turns and stored as uint32
// fixed point).  Per (sample, k) the phase a + k b is formed exactly in
// wrapping 32-bit integer arithmetic, so its error is at most (1 + k) 2^-33
// turns; the final sine/cosine of the reduced angle (in [-pi, pi)) runs in
// FP32 on the special-function unit.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

// ------------------------------------------------------------------ z_ref
// Mean of z_l = p_z + (tx_z + rx_z)/2 over all samples, i.e.
// mean(p_z) + (mean(tx_z) + mean(rx_z))/2.  Every block sums a fixed slice of
// the positions in a fixed order and the last block to finish adds the block
// sums in index order, so the result is the same bits on every run.  The
// finishing thread also resolves Z_c = z_scene - z_ref of Eq. 12 once for
// all samples (its reciprocal term 1 / (4 Z_c), and the check Z_c > 0).
// Block 0 resets the occupied-window accumulators of the header.
constexpr int kZrefThreads = 256;
constexpr int kZrefMaxBlocks = 128;   // <= kZrefThreads (the last block loads one sum per thread)

__device__ __forceinline__ void resolve_zref(double z_ref, double z_scene, int compensate, WsHeader *hdr) {
    hdr->z_ref = z_ref;
    const double Zc = z_scene - z_ref;
    if (compensate && !(Zc > 0.0)) atomicOr(&hdr->error, kErrGeometry);
    hdr->inv_4zc = (compensate && Zc > 0.0) ? 1.0 / (4.0 * Zc) : 0.0;
    hdr->zc = (compensate && Zc > 0.0) ? Zc : 0.0;
}

// Classes of the Tx/Rx pairs for the grouped gridding: pairs whose x offsets
// sum to the same value (tx_x + rx_x, compared exactly) put their virtual
// elements at the same x' for every position (Eq. 3).  Classes are numbered
// in order of first appearance; the tables hold the class of each pair, the
// start of each class in the member list and the members in ascending pair
// order.  One block, every thread of it (pairs <= kMaxPairsGrouped <= threads).
static_assert(kMaxPairsGrouped <= kZrefThreads, "one thread per pair");

__device__ void pair_classes(const double *__restrict__ tx, const double *__restrict__ rx, int T, int R,
                             int *cls, WsHeader *hdr) {
    __shared__ double xo[kMaxPairsGrouped];
    __shared__ int pc[kMaxPairsGrouped];
    const int TR = T * R, tid = threadIdx.x;
    if (TR > kMaxPairsGrouped) {
        if (tid == 0) hdr->n_classes = 0;
        return;
    }
    if (tid < TR) xo[tid] = tx[3 * (tid / R)] + rx[3 * (tid % R)];
    __syncthreads();
    // representative: the first pair with the same offset; the class number
    // is the count of representatives before it
    int rep = tid;
    if (tid < TR)
        for (int q = 0; q < tid; ++q)
            if (xo[q] == xo[tid]) {
                rep = q;
                break;
            }
    __syncthreads();
    if (tid < TR) pc[tid] = rep == tid ? 1 : 0;   // representative flags
    __syncthreads();
    int c = 0, n_cls = 0;
    if (tid < TR) {
        for (int q = 0; q < TR; ++q) {
            n_cls += pc[q];
            if (q < rep) c += pc[q];
        }
    }
    __syncthreads();
    if (tid < TR) pc[tid] = c;
    __syncthreads();
    int *pclass = cls, *start = cls + TR, *members = cls + 2 * TR + 1;
    if (tid < TR) {
        // members of the classes before c, then the pairs of class c before this one
        int pos = 0;
        for (int q = 0; q < TR; ++q) pos += (pc[q] < c) || (pc[q] == c && q < tid);
        members[pos] = tid;
        pclass[tid] = c;
        if (rep == tid) {
            int before = 0;
            for (int q = 0; q < TR; ++q) before += pc[q] < c;
            start[c] = before;
        }
        if (tid == 0) {
            start[n_cls] = TR;
            hdr->n_classes = n_cls;
        }
    }
}

struct ZrefArgs {
    const double *pos, *tx, *rx;
    int P, T, R, given, compensate, pad;
    double z_given, z_scene;
    double *partials;
    int *cls;
    WsHeader *hdr;
};

// bid / nb: this block's index and the block count of this scan
__device__ __forceinline__ void zref_body(const ZrefArgs &a, int bid, int nb) {
    __shared__ double red[kZrefThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int P = a.P;
    if (bid == 0) {
        if (tid == 0) {
            a.hdr->u_min = a.hdr->v_min = 0x7fffffff;
            a.hdr->u_max = a.hdr->v_max = -0x7fffffff - 1;
            if (a.given) resolve_zref(a.z_given, a.z_scene, a.compensate, a.hdr);
        }
        pair_classes(a.tx, a.rx, a.T, a.R, a.cls, a.hdr);
    }
    if (a.given) return;
    const int per = (P + nb - 1) / nb;
    const int p0 = bid * per, p1 = min(P, p0 + per);
    double acc = 0.0;
    for (int p = p0 + tid; p < p1; p += kZrefThreads) acc += a.pos[3 * p + 2];
    red[tid] = acc;
    __syncthreads();
    for (int h = kZrefThreads / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        a.partials[bid] = red[0];
        __threadfence();
        last = atomicAdd(&a.hdr->zref_done, 1) == nb - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: the block sums loaded in parallel (nb <= 256), then the
    // same fixed-order tree as above
    __threadfence();
    red[tid] = tid < nb ? ((volatile double *)a.partials)[tid] : 0.0;
    __syncthreads();
    for (int h = kZrefThreads / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        double st = 0.0, sr = 0.0;
        for (int t = 0; t < a.T; ++t) st += a.tx[3 * t + 2];
        for (int r = 0; r < a.R; ++r) sr += a.rx[3 * r + 2];
        const double mean_p = P > 0 ? __ddiv_rn(red[0], (double)P) : 0.0;
        const double mean_tr = __dmul_rn(0.5, __dadd_rn(__ddiv_rn(st, (double)a.T), __ddiv_rn(sr, (double)a.R)));
        resolve_zref(__dadd_rn(mean_p, mean_tr), a.z_scene, a.compensate, a.hdr);
    }
}

__global__ void __launch_bounds__(kZrefThreads) zref_kernel(const __grid_constant__ ZrefArgs a) {
    zref_body(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kZrefThreads) zref_multi(const __grid_constant__ BatchTable<ZrefArgs> t) {
    __shared__ ZrefArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    zref_body(sa, bid, nb);
}

static int zref_describe(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                         ZrefArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.pos = pos;
    a.tx = tx;
    a.rx = rx;
    a.P = p.shape.n_pos;
    a.T = p.shape.n_tx;
    a.R = p.shape.n_rx;
    a.given = p.zref_given ? 1 : 0;
    a.compensate = p.opt.compensate;
    a.pad = 0;
    a.z_given = p.z_ref;
    a.z_scene = p.z_scene;
    a.partials = reinterpret_cast<double *>(w + p.off_partials);
    a.cls = reinterpret_cast<int *>(w + p.off_cls);
    a.hdr = reinterpret_cast<WsHeader *>(w);
    // about one position per thread, at most kZrefMaxBlocks blocks
    int blocks = (p.shape.n_pos + kZrefThreads - 1) / kZrefThreads;
    blocks = blocks < 1 ? 1 : (blocks > kZrefMaxBlocks ? kZrefMaxBlocks : blocks);
    return p.zref_given ? 1 : blocks;
}

cudaError_t launch_zref(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                        cudaStream_t s) {
    ZrefArgs a;
    const int blocks = zref_describe(p, ws, pos, tx, rx, a);
    zref_kernel<<<blocks, kZrefThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_zref_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<ZrefArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n, 0);
    for (int i = 0; i < n; ++i)
        blocks[i] = zref_describe(r[i].plan->p, r[i].workspace, r[i].pos, r[i].tx, r[i].rx, args[i]);
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int, const BatchTable<ZrefArgs> &t, int total) {
                             zref_multi<<<total, kZrefThreads, 0, s>>>(t);
                             return cudaGetLastError();
                         });
}

// ------------------------------------------------------------------ geometry
struct GeomArgs {
    const double *pos, *tx, *rx;
    int T, R, P;
    int L;                               // below 2^30 (plan limit)
    double x_c, y_c, inv_dx2, inv_dy2;   // 2 / dx: cells of the 2M grid per metre
    int compensate;
    double half_w;
    int mrx, mry, nbx;
    double f0_over_c32, df_over_c32;   // f0 / c and df / c times 2^32 (turns per metre, fixed point)
    WsHeader *hdr;
    int *counts;
    int *offsets, *cursor;   // bin scan (last block)
    int n_bins, w;
    int *binid;
    SampleRec *rec;
    uint2 *phase;
    // grouped gridding: bins hold groups (class, position) instead of samples
    int grouped, G;
    const int *cls;          // pair classes (see pair_classes)
    GroupRec *grec;
};

// A phase given as turns x 2^32 -> 32-bit fixed-point turns: the low 32 bits
// of the nearest integer are the phase modulo one turn (the scaling by 2^32
// is exact, so this equals rounding frac(turns) 2^32).  Beyond 2^63 the
// fraction is taken first.
__device__ __forceinline__ uint32_t turns32_to_fixed(double t32) {
    if (fabs(t32) < 9.0e18) return (uint32_t)(unsigned long long)llrint(t32);
    const double f = t32 * 2.3283064365386963e-10;   // turns
    return (uint32_t)(unsigned long long)llrint((f - floor(f)) * 4294967296.0);
}

__device__ __forceinline__ void box_reduce(int umin, int umax, int vmin, int vmax, WsHeader *hdr) {
    for (int o = 16; o > 0; o >>= 1) {
        umin = min(umin, __shfl_xor_sync(0xffffffffu, umin, o));
        umax = max(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if ((threadIdx.x & 31) == 0 && umin <= umax) {
        atomicMin(&hdr->u_min, umin);
        atomicMax(&hdr->u_max, umax);
        atomicMin(&hdr->v_min, vmin);
        atomicMax(&hdr->v_max, vmax);
    }
}

// Returns the sample's bin (-1 when it is not binned); the caller counts it.
// With bin_it false (grouped gridding) the sample is neither binned nor part
// of the occupied window: its group is.
__device__ int geometry_one(const GeomArgs &a, int l, int &umin, int &umax, int &vmin, int &vmax, bool bin_it) {
    const int tr = l / a.P, p = l - tr * a.P;
    const int t = tr / a.R, r = tr - t * a.R;
    const double px = a.pos[3 * p], py = a.pos[3 * p + 1], pz = a.pos[3 * p + 2];
    // Tx / Rx absolute positions (Eq. 2 geometry)
    const double xT = px + a.tx[3 * t], yT = py + a.tx[3 * t + 1], zT = pz + a.tx[3 * t + 2];
    const double xR = px + a.rx[3 * r], yR = py + a.rx[3 * r + 1], zR = pz + a.rx[3 * r + 2];
    // Eq. 3-4: virtual element at the midpoint, separations, plane offset
    const double xv = __dmul_rn(0.5, __dadd_rn(xT, xR)), yv = __dmul_rn(0.5, __dadd_rn(yT, yR));
    const double zl = __dmul_rn(0.5, __dadd_rn(zT, zR));
    const double ddx = __dsub_rn(xR, xT), ddy = __dsub_rn(yR, yT);
    const double z_ref = a.hdr->z_ref, inv_4zc = a.hdr->inv_4zc;
    if (!(isfinite(xv) && isfinite(yv) && isfinite(zl))) {
        atomicOr(&a.hdr->error, kErrNonfinite);
        if (bin_it) a.binid[l] = -1;
        return -1;
    }
    // residual of the round trip over 2 R_0 (Z_c <= 0 was flagged once when
    // z_ref was resolved; beta is then 0).  Every FP64 operation of the
    // per-sample geometry is an explicitly rounded one (no fused
    // multiply-adds left to the compiler), so that every kernel instance that
    // inlines it -- one scan or a fused batch -- computes the same bits.
    double beta = 0.0;
    if (a.compensate == 1 && inv_4zc > 0.0) {
        // Eq. 12 with +z toward the scene: beta = -2 d^z + (d^x^2 + d^y^2) / (4 Z_c)
        const double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
        beta = __dadd_rn(__dmul_rn(-2.0, __dsub_rn(zl, z_ref)), __dmul_rn(d2, inv_4zc));
    } else if (a.compensate == 2 && inv_4zc > 0.0) {
        // Eq. 5 at the scene centre (x_c, y_c, z_ref + Z_c), Z_0 - z = -Z_c:
        //   beta = -2 Z_c d^z / R_0 + (d^x^2 + d^y^2 + 4 d^z^2) / (4 R_0)
        //          - [((x' - x_c) d^x + (y' - y_c) d^y)^2 + 4 Z_c^2 d^z^2] / (4 R_0^3)
        const double Zc = a.hdr->zc, dz = __dsub_rn(zl, z_ref);
        const double ax = __dsub_rn(xv, a.x_c), ay = __dsub_rn(yv, a.y_c);
        const double R0 = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(Zc, Zc)));
        const double cross = __dadd_rn(__dmul_rn(ax, ddx), __dmul_rn(ay, ddy));
        const double dz2 = __dmul_rn(dz, dz);
        const double t1 = __ddiv_rn(__dmul_rn(__dmul_rn(-2.0, Zc), dz), R0);
        const double t2 = __ddiv_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(4.0, dz2)),
            __dmul_rn(4.0, R0));
        const double num3 = __dadd_rn(__dmul_rn(cross, cross), __dmul_rn(__dmul_rn(4.0, __dmul_rn(Zc, Zc)), dz2));
        const double t3 = __ddiv_rn(num3, __dmul_rn(__dmul_rn(4.0, R0), __dmul_rn(R0, R0)));
        beta = __dsub_rn(__dadd_rn(t1, t2), t3);
    }
    // position on the 2M-point periodic grid, in cells
    const double gx = __dmul_rn(__dsub_rn(xv, a.x_c), a.inv_dx2);
    const double gy = __dmul_rn(__dsub_rn(yv, a.y_c), a.inv_dy2);
    const double u0d = ceil(__dsub_rn(gx, a.half_w)), v0d = ceil(__dsub_rn(gy, a.half_w));
    const double fx = __dsub_rn(gx, u0d), fy = __dsub_rn(gy, v0d);
    // occupied window; a sample absurdly far away (beyond 1e9 cells) makes the
    // window the whole grid
    const bool ufar = fabs(u0d) > 1.0e9, vfar = fabs(v0d) > 1.0e9;
    if (bin_it) {
        umin = ufar ? -1073741824 : (int)u0d;
        umax = ufar ? 1073741823 : (int)u0d;
        vmin = vfar ? -1073741824 : (int)v0d;
        vmax = vfar ? 1073741823 : (int)v0d;
    }
    // wrap into [0, M_r) (M_r is a power of two; beyond 2^62 cells the
    // position is meaningless and is put at cell 0)
    const long long u0l = fabs(u0d) < 4.0e18 ? (long long)u0d : 0;
    const long long v0l = fabs(v0d) < 4.0e18 ? (long long)v0d : 0;
    const int u0 = (int)(u0l & (a.mrx - 1)), v0 = (int)(v0l & (a.mry - 1));
    SampleRec rc;
    rc.u0 = u0;
    rc.v0 = v0;
    rc.fx = (float)fx;
    rc.fy = (float)fy;
    a.rec[l] = rc;
    // Eq. 11 phase k beta = 2 pi f beta / c in turns: f0 beta/c + k df beta/c
    a.phase[l] = make_uint2(turns32_to_fixed(a.f0_over_c32 * beta), turns32_to_fixed(a.df_over_c32 * beta));
    if (!bin_it) return -1;
    const int bin = (rc.v0 / kBin) * a.nbx + rc.u0 / kBin;
    a.binid[l] = bin;
    return bin;
}

// Group g = (class c, position p) of the grouped gridding: the class's shared
// x' (computed as its first member's sample does) gives the x cell; the
// lowest and highest first y cell of its members (computed as their samples
// do) give the group's y extent.  Returns the group's bin (-1: no group).
__device__ int group_one(const GeomArgs &a, int g, int &umin, int &umax, int &vmin, int &vmax, int &vspan) {
    const int TR = a.T * a.R;
    const int c = g / a.P, p = g - c * a.P;
    if (c >= a.hdr->n_classes) {
        a.binid[g] = -1;
        return -1;
    }
    const int *start = a.cls + TR, *members = a.cls + 2 * TR + 1;
    const int m_beg = start[c], m_end = start[c + 1];
    const int m0 = members[m_beg], t0 = m0 / a.R, r0 = m0 - t0 * a.R;
    const double px = a.pos[3 * p], py = a.pos[3 * p + 1];
    const double xv = __dmul_rn(0.5, __dadd_rn(__dadd_rn(px, a.tx[3 * t0]), __dadd_rn(px, a.rx[3 * r0])));
    bool ok = isfinite(xv);
    double vlo = 0.0, vhi = 0.0;
    for (int m = m_beg; m < m_end; ++m) {
        const int tr = members[m], t = tr / a.R, r = tr - t * a.R;
        const double yv = __dmul_rn(0.5, __dadd_rn(__dadd_rn(py, a.tx[3 * t + 1]), __dadd_rn(py, a.rx[3 * r + 1])));
        ok = ok && isfinite(yv);
        const double v0d = ceil(__dsub_rn(__dmul_rn(__dsub_rn(yv, a.y_c), a.inv_dy2), a.half_w));
        vlo = m == m_beg ? v0d : fmin(vlo, v0d);
        vhi = m == m_beg ? v0d : fmax(vhi, v0d);
    }
    if (!ok) {
        atomicOr(&a.hdr->error, kErrNonfinite);
        a.binid[g] = -1;
        return -1;
    }
    const double gx = __dmul_rn(__dsub_rn(xv, a.x_c), a.inv_dx2);
    const double u0d = ceil(__dsub_rn(gx, a.half_w));
    const bool ufar = fabs(u0d) > 1.0e9, vfar = fabs(vlo) > 1.0e9 || fabs(vhi) > 1.0e9;
    umin = ufar ? -1073741824 : (int)u0d;
    umax = ufar ? 1073741823 : (int)u0d;
    vmin = vfar ? -1073741824 : (int)vlo;
    vmax = vfar ? 1073741823 : (int)vhi;
    const long long u0l = fabs(u0d) < 4.0e18 ? (long long)u0d : 0;
    const long long v0l = fabs(vlo) < 4.0e18 ? (long long)vlo : 0;
    GroupRec gr;
    gr.u0 = (int)(u0l & (a.mrx - 1));
    gr.v0min = (int)(v0l & (a.mry - 1));
    gr.fx = (float)__dsub_rn(gx, u0d);
    gr.vspan = vfar ? 0 : (int)fmin(vhi - vlo, (double)(a.mry - 1));
    a.grec[g] = gr;
    vspan = gr.vspan;
    const int bin = (gr.v0min / kBin) * a.nbx + gr.u0 / kBin;
    a.binid[g] = bin;
    return bin;
}

__device__ void scan_bins(const int *counts, int *__restrict__ offsets, int *__restrict__ cursor, int n,
                          WsHeader *hdr, int w, int mrx, int mry, int *warp_tot);

__device__ __forceinline__ void geometry_body(const GeomArgs &a, int bid, int nb) {
    __shared__ int warp_tot[32];
    __shared__ bool last;
    const int l = bid * blockDim.x + threadIdx.x;
    int bumin = 0x7fffffff, bumax = -0x7fffffff - 1, bvmin = 0x7fffffff, bvmax = -0x7fffffff - 1;
    int bin = -1, vspan = 0;
    if (l < a.L)
        bin = geometry_one(a, l, bumin, bumax, bvmin, bvmax, !a.grouped);
    else if (a.grouped && l - a.L < a.G)
        bin = group_one(a, l - a.L, bumin, bumax, bvmin, bvmax, vspan);
    if (a.grouped) {   // the largest group span, one atomic per warp
        for (int o = 16; o > 0; o >>= 1) vspan = max(vspan, __shfl_xor_sync(0xffffffffu, vspan, o));
        if ((threadIdx.x & 31) == 0 && vspan > 0) atomicMax(&a.hdr->vspan_max, vspan);
    }
    // neighbouring samples share bins: one atomic per distinct bin of the warp
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&a.counts[bin], __popc(grp));
    box_reduce(bumin, bumax, bvmin, bvmax, a.hdr);
    // the last block to finish turns the bin counts into offsets
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&a.hdr->geom_done, 1) == nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    scan_bins(a.counts, a.offsets, a.cursor, a.n_bins, a.hdr, a.w, a.mrx, a.mry, warp_tot);
}

__global__ void __launch_bounds__(256) geometry_kernel(const __grid_constant__ GeomArgs a) {
    geometry_body(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) geometry_multi(const __grid_constant__ BatchTable<GeomArgs> t) {
    __shared__ GeomArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    geometry_body(sa, bid, nb);
}

static int geometry_describe(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                             GeomArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.pos = pos;
    a.tx = tx;
    a.rx = rx;
    a.T = p.shape.n_tx;
    a.R = p.shape.n_rx;
    a.P = p.shape.n_pos;
    a.L = (int)p.L;
    a.x_c = p.grid.x0 + (p.grid.nx / 2) * p.grid.dx;
    a.y_c = p.grid.y0 + (p.grid.ny / 2) * p.grid.dy;
    a.inv_dx2 = (double)p.mrx / ((double)p.mx * p.grid.dx);
    a.inv_dy2 = (double)p.mry / ((double)p.my * p.grid.dy);
    a.compensate = p.opt.compensate;
    a.half_w = 0.5 * p.w;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.f0_over_c32 = p.shape.f0_hz / kC0 * 4294967296.0;
    a.df_over_c32 = p.shape.df_hz / kC0 * 4294967296.0;
    a.hdr = reinterpret_cast<WsHeader *>(w);
    a.counts = reinterpret_cast<int *>(w + p.off_counts);
    a.offsets = reinterpret_cast<int *>(w + p.off_offsets);
    a.cursor = reinterpret_cast<int *>(w + p.off_cursor);
    a.n_bins = (int)p.n_bins;
    a.w = p.w;
    a.binid = reinterpret_cast<int *>(w + p.off_binid);
    a.rec = reinterpret_cast<SampleRec *>(w + p.off_rec);
    a.phase = reinterpret_cast<uint2 *>(w + p.off_phase);
    a.grouped = p.grouped ? 1 : 0;
    a.G = (int)p.G;
    a.cls = reinterpret_cast<const int *>(w + p.off_cls);
    a.grec = reinterpret_cast<GroupRec *>(w + p.off_grec);
    const long long threads = p.L + (p.grouped ? p.G : 0);
    return (int)((threads + 255) / 256);
}

cudaError_t launch_geometry(const Plan &p, void *ws, const double *pos, const double *tx, const double *rx,
                            cudaStream_t s) {
    GeomArgs a;
    const int blocks = geometry_describe(p, ws, pos, tx, rx, a);
    geometry_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_geometry_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<GeomArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n, 0);
    for (int i = 0; i < n; ++i)
        blocks[i] = geometry_describe(r[i].plan->p, r[i].workspace, r[i].pos, r[i].tx, r[i].rx, args[i]);
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int, const BatchTable<GeomArgs> &t, int total) {
                             geometry_multi<<<total, 256, 0, s>>>(t);
                             return cudaGetLastError();
                         });
}

// ------------------------------------------------------------------ bin scan
// Occupied window of one axis from the min / max first cell: cells
// lo .. lo + len - 1 (mod m) can receive a tap.
__device__ __forceinline__ void finish_window(int vmin, int vmax, int w, int m, int *lo, int *len) {
    if (vmin > vmax) {          // no sample
        *lo = 0;
        *len = 0;
        return;
    }
    const long long span = (long long)vmax - vmin + w;
    if (span >= m) {
        *lo = 0;
        *len = m;
        return;
    }
    int l0 = vmin % m;
    if (l0 < 0) l0 += m;
    *lo = l0;
    *len = (int)span;
}

// Exclusive prefix sum of the bin counts by one block (the last block of the
// geometry pass), in rounds of blockDim.x x kScanPer bins: thread t loads its
// kScanPer consecutive bins with 16-byte loads from L2 (the counts were
// built by atomics of other blocks), the block scans the per-thread sums with
// warp shuffles, and every thread writes its bins' offsets (also the scatter
// cursors); the running total carries to the next round.  The bin count is
// a multiple of 4.  Thread 0 finalises the occupied window and the
// binned-sample count.
constexpr int kScanPer = 16;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    return x - v + (warp > 0 ? warp_tot[warp - 1] : 0);
}

__device__ void scan_bins(const int *counts, int *__restrict__ offsets, int *__restrict__ cursor, int n,
                          WsHeader *hdr, int w, int mrx, int mry, int *warp_tot) {
    int carry = 0;
    for (int base = 0; base < n; base += blockDim.x * kScanPer) {
        const int b0 = base + threadIdx.x * kScanPer;
        int4 c[kScanPer / 4];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) {
            c[q] = b0 + 4 * q < n ? __ldcg(reinterpret_cast<const int4 *>(counts + b0 + 4 * q)) : make_int4(0, 0, 0, 0);
            sum += c[q].x + c[q].y + c[q].z + c[q].w;
        }
        int total;
        int run = carry + block_exclusive_scan(sum, warp_tot, total);
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) {
            if (b0 + 4 * q >= n) break;
            int4 o;
            o.x = run;
            o.y = o.x + c[q].x;
            o.z = o.y + c[q].y;
            o.w = o.z + c[q].z;
            run = o.w + c[q].w;
            *reinterpret_cast<int4 *>(offsets + b0 + 4 * q) = o;
            *reinterpret_cast<int4 *>(cursor + b0 + 4 * q) = o;
        }
        carry += total;
        __syncthreads();   // warp_tot is reused by the next round
    }
    if (threadIdx.x == 0) {
        offsets[n] = carry;
        hdr->n_valid = carry;
        volatile WsHeader *vh = hdr;
        finish_window(vh->u_min, vh->u_max, w, mrx, &hdr->u_lo, &hdr->u_len);
        finish_window(vh->v_min, vh->v_max, w, mry, &hdr->v_lo, &hdr->v_len);
    }
}

// ------------------------------------------------------------------ bin scatter
// Each sample takes a slot of its bin: the lanes of a warp that share a bin
// reserve their slots with one atomic and take them in lane order (the
// in-bin order is made deterministic afterwards by the in-bin sort).
struct ScatterArgs {
    int L, pad;
    const int *binid;
    int *cursor, *perm;
};

__device__ __forceinline__ void bin_scatter_body(const ScatterArgs &a, int bid) {
    const int l = bid * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int b = l < a.L ? a.binid[l] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (b >= 0 && lane == leader) base = atomicAdd(&a.cursor[b], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b >= 0) a.perm[base + __popc(grp & ((1u << lane) - 1u))] = l;
}

__global__ void __launch_bounds__(256) bin_scatter_kernel(const __grid_constant__ ScatterArgs a) {
    bin_scatter_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(256) bin_scatter_multi(const __grid_constant__ BatchTable<ScatterArgs> t) {
    __shared__ ScatterArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    bin_scatter_body(sa, bid);
}

static int bin_scatter_describe(const Plan &p, void *ws, ScatterArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    const long long items = p.grouped ? p.G : p.L;   // groups or samples
    a.L = (int)items;
    a.pad = 0;
    a.binid = reinterpret_cast<const int *>(w + p.off_binid);
    a.cursor = reinterpret_cast<int *>(w + p.off_cursor);
    a.perm = reinterpret_cast<int *>(w + p.off_perm);
    return (int)((items + 255) / 256);
}

cudaError_t launch_bin_scatter(const Plan &p, void *ws, cudaStream_t s) {
    ScatterArgs a;
    const int blocks = bin_scatter_describe(p, ws, a);
    bin_scatter_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<ScatterArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n, 0);
    for (int i = 0; i < n; ++i) blocks[i] = bin_scatter_describe(r[i].plan->p, r[i].workspace, args[i]);
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int, const BatchTable<ScatterArgs> &t, int total) {
                             bin_scatter_multi<<<total, 256, 0, s>>>(t);
                             return cudaGetLastError();
                         });
}

// ------------------------------------------------------------------ compensate and in-bin order
// One launch with two kinds of blocks that run side by side.  The first
// n_sort blocks finish the binning, one warp per bin: the in-bin sort and the
// per-sample gridding records.  The other blocks apply Eq. 11 to every
// sample.  The compensation is HBM-bound and the sort latency-bound, so the
// sort hides under the compensation; neither reads what the other writes.

// -- in-bin sort and gridding records
// The scatter filled each bin in the arrival order of its atomics.  A rank
// sort puts the samples of a bin of up to kSortBinCap samples in ascending
// sample order (a fixed summation order makes the image bit-reproducible;
// larger bins keep the arrival order, which is still correct, only the last
// bits of the image can then vary between runs).  Then, per sample in that
// order: its in-bin offset and sample index, and per axis w + 3 weight quads
// (quad q = the Gaussian weights exp(-kappa (f - tap)^2) of taps q-3 .. q,
// zero outside 0..w-1), consecutive lanes writing consecutive 16-byte entries.
constexpr int kSortBinCap = 256;
constexpr int kPrepWarps = 8;

// Gaussian weights exp(-kappa (f - tap)^2) of taps q-3 .. q (zero outside
// 0 .. w-1): the four weights a 4-cell block needs when it starts q - 3 cells
// after the first tap.
__device__ __forceinline__ float4 weight_quad(float f, int q, int w, float kappa) {
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int tap = q - 3 + i;
        const float dlt = f - (float)tap;
        v[i] = (tap >= 0 && tap < w) ? expf(-kappa * dlt * dlt) : 0.f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

// Rank sort of one bin's entries (perm[beg .. beg + n)) into ascending order
// in shared memory when the bin holds at most kSortBinCap of them (larger
// bins keep the arrival order: still correct, only the last bits of the
// image can then vary between runs).  Returns whether it sorted.
__device__ bool sort_bin(int *pp, int n, int *keys, int *sorted) {
    const int lane = threadIdx.x & 31;
    if (n > kSortBinCap) return false;
    for (int i = lane; i < n; i += 32) keys[i] = pp[i];
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const int ki = keys[i];
        int rank = 0;   // #{j : key_j < key_i}; the entries are distinct
        for (int j = 0; j < n; ++j) rank += keys[j] < ki;
        sorted[rank] = ki;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) pp[i] = sorted[i];
    return true;
}

// Grouped gridding: one bin of groups in ascending group order, and per group
// in that order its in-bin offsets with its index, and its w + 3 x weight quads.
__device__ void sort_and_weigh_group_bin(int b, const int *__restrict__ offsets, int *__restrict__ perm,
                                         const GroupRec *__restrict__ grec, int w, float kappa,
                                         int2 *__restrict__ gdd, float4 *__restrict__ gxq, int4 *__restrict__ goff,
                                         const SampleRec *__restrict__ rec, const int *__restrict__ cls, int TR,
                                         int P, int mry, int *keys, int *sorted) {
    const int lane = threadIdx.x & 31;
    const int beg = offsets[b], n = offsets[b + 1] - beg;
    if (n == 0) return;
    int *pp = perm + beg;
    const bool small = sort_bin(pp, n, keys, sorted);
    const int nq = w + 3;
    const int total = n * nq;
    for (int e = lane; e < total; e += 32) {
        const int sl = e / nq, q = e - sl * nq;
        const int g = small ? sorted[sl] : pp[sl];
        const GroupRec r = grec[g];
        if (q == 0) {
            gdd[beg + sl] = make_int2((r.u0 & 3) | ((r.v0min & 3) << 2), g);
            // the members' first y cells above the group's lowest, 16 bits each
            const int c = g / P, pp = g - c * P;
            const int *start = cls + TR, *members = cls + 2 * TR + 1;
            unsigned o[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            for (int m = start[c]; m < start[c + 1]; ++m) {
                const int k = m - start[c];
                const unsigned off = (unsigned)((rec[members[m] * P + pp].v0 - r.v0min) & (mry - 1)) & 0xffffu;
                o[k >> 1] |= off << (16 * (k & 1));
            }
            goff[2 * (beg + sl)] = make_int4((int)o[0], (int)o[1], (int)o[2], (int)o[3]);
            goff[2 * (beg + sl) + 1] = make_int4((int)o[4], (int)o[5], (int)o[6], (int)o[7]);
        }
        gxq[(long long)(beg + sl) * nq + q] = weight_quad(r.fx, q, w, kappa);
    }
}

__device__ void sort_and_weigh_bin(int b, const int *__restrict__ offsets, int *__restrict__ perm,
                                   const SampleRec *__restrict__ rec, int w, float kappa, int2 *__restrict__ dd,
                                   float4 *__restrict__ wrec, int *keys, int *sorted) {
    const int lane = threadIdx.x & 31;
    const int beg = offsets[b], n = offsets[b + 1] - beg;
    if (n == 0) return;
    int *pp = perm + beg;
    const bool small = sort_bin(pp, n, keys, sorted);
    const int nq = w + 3, rq = 2 * nq + 1;
    const int total = n * rq;
    for (int e = lane; e < total; e += 32) {
        const int sl = e / rq, ent = e - sl * rq;
        const int l = small ? sorted[sl] : pp[sl];
        const SampleRec r = rec[l];
        float4 out;
        if (ent == 0) {
            const int d = (r.u0 & 3) | ((r.v0 & 3) << 2);
            dd[beg + sl] = make_int2(d, l);
            out = make_float4(__int_as_float(d), __int_as_float(l), 0.f, 0.f);
        } else {
            const int q = (ent - 1) % nq;                 // quad q = taps q-3 .. q
            out = weight_quad((ent - 1) < nq ? r.fx : r.fy, q, w, kappa);
        }
        wrec[(long long)(beg + sl) * rq + ent] = out;
    }
}

// Tensor-core gridding: one bin in ascending sample order, and per sample in
// that order a 16-byte record (sample index, first cell u0 | v0 << 16, cell
// fractions fx, fy).
__device__ void sort_and_record_bin_tc(int b, const int *__restrict__ offsets, int *__restrict__ perm,
                                       const SampleRec *__restrict__ rec, int4 *__restrict__ trec, int *keys,
                                       int *sorted) {
    const int lane = threadIdx.x & 31;
    const int beg = offsets[b], n = offsets[b + 1] - beg;
    if (n == 0) return;
    int *pp = perm + beg;
    const bool small = sort_bin(pp, n, keys, sorted);
    for (int sl = lane; sl < n; sl += 32) {
        const int l = small ? sorted[sl] : pp[sl];
        const SampleRec r = rec[l];
        trec[beg + sl] = make_int4(l, (r.u0 & 0xffff) | (r.v0 << 16), __float_as_int(r.fx), __float_as_int(r.fy));
    }
}

// -- compensation (Eq. 11)
// One warp per group of kCompUnroll samples and one 64-frequency group g:
// each lane reads two frequencies of each sample of the group (the loads of
// the group are issued together and coalesced), rotates them by
// exp(+j 2 pi (a + k b)) and writes s_hat in original sample order,
// s_hat[g][l][0..63] (512 contiguous bytes per sample; frequencies past Nk
// are written as zero).
constexpr int kCompUnroll = 4;

template <int DT>
__device__ __forceinline__ float2 load_echo(const void *__restrict__ echo_v, long long e, float scale) {
    if (DT == MMSAR_ECHO_C64) {
        return __ldg(reinterpret_cast<const float2 *>(echo_v) + e);
    } else if (DT == MMSAR_ECHO_F16X2_SCALED) {
        const __half2 h = reinterpret_cast<const __half2 *>(echo_v)[e];
        float2 v = __half22float2(h);
        return make_float2(v.x * scale, v.y * scale);
    } else {
        const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162 *>(echo_v)[e];
        float2 v = __bfloat1622float2(h);
        return make_float2(v.x * scale, v.y * scale);
    }
}

// Two adjacent complex samples (pair index e2 = element index / 2): 16 bytes
// of complex64 or 8 bytes of scaled FP16 / BF16 pairs.
template <int DT>
__device__ __forceinline__ void load_echo2(const void *__restrict__ echo_v, long long e2, float scale, float2 &v0,
                                           float2 &v1) {
    if (DT == MMSAR_ECHO_C64) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(echo_v) + e2);
        v0 = make_float2(t.x, t.y);
        v1 = make_float2(t.z, t.w);
    } else {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(echo_v) + e2);
        float2 a, b;
        if (DT == MMSAR_ECHO_F16X2_SCALED) {
            a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
            b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        } else {
            a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.x));
            b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.y));
        }
        v0 = make_float2(a.x * scale, a.y * scale);
        v1 = make_float2(b.x * scale, b.y * scale);
    }
}

// exp(+j 2 pi turns / 2^32) applied to v; the angle is already reduced to
// [-pi, pi), where the hardware sine and cosine (absolute error ~4e-7) are
// accurate enough
__device__ __forceinline__ float2 rotate_turns(float2 v, uint32_t turns) {
    const float ang = (float)(int32_t)turns * 1.4629180792671596e-09f;   // 2 pi turns / 2^32
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    return cmul(v, make_float2(cs, sn));
}

struct PrepTailArgs {
    // in-bin order
    int n_bins, n_sort_blocks;
    const int *offsets;
    int *perm;
    const SampleRec *rec;
    int w;
    float kappa;
    int2 *dd;
    float4 *wrec;
    // grouped gridding: group records, their sorted offsets and x quads, and
    // per sample (original order) a header with the first-y-cell offset
    // within its group followed by its y quads
    int grouped, n_yrec_blocks, P, R, TR, mry;
    const GroupRec *grec;
    const int *cls;
    int2 *gdd;
    int4 *goff;
    float4 *gxq, *yq;
    // tensor-core gridding: compact records (bin order) instead of the above
    int tc;
    int4 *trec;
    // compensation
    const void *echo;
    const float *scale;
    const uint2 *phase;
    int Nk, L, chunk_blocks;
    int *err;
    float2 *shat;
    // split output (tensor-core gridding): s_hat 2^a as FP16 hi / lo planes
    // [g][L][2][128 halves] (shat reinterpreted), one exponent a per sample
    // [L], and the max of 127 - a over all samples (one int)
    signed char *sexp;
    int *aref;
};

// Power-of-two normalisation of a sample's row: a such that m 2^a lies in
// [2^13, 2^14) for its largest magnitude m (127 for an all-zero row, clamped
// to +-120 otherwise).
__device__ __forceinline__ int norm_exponent(float m) {
    if (!(m > 0.f) || !isfinite(m)) return m > 0.f ? -120 : 127;
    int e;
    frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
    const int a = 14 - e;
    return a < -120 ? -120 : (a > 120 ? 120 : a);
}

// FP16 hi / lo split of two values scaled by 2^a (exact scaling): (hi, lo) half2 pairs
__device__ __forceinline__ void split2(float x, float y, float sc, __half2 &hi, __half2 &lo) {
    const float xs = x * sc, ys = y * sc;
    hi = __floats2half2_rn(xs, ys);
    const float2 h = __half22float2(hi);
    lo = __floats2half2_rn(xs - h.x, ys - h.y);
}

// VEC: lane l takes the adjacent frequencies 64 g + 2 l and 64 g + 2 l + 1
// (one 16-byte or 8-byte load, one 16-byte store per sample; Nk even and the
// echo aligned); otherwise 64 g + l and 64 g + 32 + l.
template <int DT, bool VEC>
__device__ __forceinline__ void compensate_split_body(const PrepTailArgs &a, int cblk);

template <int DT, bool VEC, bool SPLIT>
__device__ __forceinline__ void compensate_body(const PrepTailArgs &a, int bid) {
    __shared__ int keys[kPrepWarps][kSortBinCap];
    __shared__ int sorted[kPrepWarps][kSortBinCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (bid < a.n_sort_blocks) {
        const int b = bid * kPrepWarps + warp;
        if (b < a.n_bins) {
            if (a.tc)
                sort_and_record_bin_tc(b, a.offsets, a.perm, a.rec, a.trec, keys[warp], sorted[warp]);
            else if (a.grouped)
                sort_and_weigh_group_bin(b, a.offsets, a.perm, a.grec, a.w, a.kappa, a.gdd, a.gxq, a.goff, a.rec,
                                         a.cls, a.TR, a.P, a.mry, keys[warp], sorted[warp]);
            else
                sort_and_weigh_bin(b, a.offsets, a.perm, a.rec, a.w, a.kappa, a.dd, a.wrec, keys[warp],
                                   sorted[warp]);
        }
        return;
    }
    if (bid < a.n_sort_blocks + a.n_yrec_blocks) {
        // grouped gridding, per sample: entry 0 holds the offset of its first
        // y cell above its group's lowest, entries 1 .. w + 3 its y quads
        const int rqy = a.w + 4;
        const long long e = (long long)(bid - a.n_sort_blocks) * blockDim.x + threadIdx.x;
        const long long l = e / rqy;
        if (l >= a.L) return;
        const int q = (int)(e - l * rqy);
        const SampleRec r = a.rec[l];
        if (q == 0) {
            const int tr = (int)(l / a.P), pp = (int)(l - (long long)tr * a.P);
            const int g = a.cls[tr] * a.P + pp;
            const int off = (r.v0 - a.grec[g].v0min) & (a.mry - 1);
            a.yq[e] = make_float4(__int_as_float(off), 0.f, 0.f, 0.f);
        } else {
            a.yq[e] = weight_quad(r.fy, q - 1, a.w, a.kappa);
        }
        return;
    }
    const int cblk = bid - a.n_sort_blocks - a.n_yrec_blocks;
    if constexpr (SPLIT) {
        compensate_split_body<DT, VEC>(a, cblk);
        return;
    }
    const int g = cblk / a.chunk_blocks, bx = cblk - g * a.chunk_blocks;
    const int Nk = a.Nk;
    const int warps = a.chunk_blocks * kPrepWarps;
    const float scale = (DT == MMSAR_ECHO_C64) ? 1.0f : *a.scale;
    bool bad = false;
    for (int g0 = (bx * kPrepWarps + warp) * kCompUnroll; g0 < a.L; g0 += warps * kCompUnroll) {
        uint2 ph[kCompUnroll];
        float2 v[kCompUnroll][2];
#pragma unroll
        for (int u = 0; u < kCompUnroll; ++u) {
            const int l = g0 + u;
            ph[u] = l < a.L ? __ldg(a.phase + l) : make_uint2(0u, 0u);
            if (VEC) {
                const int k0 = 64 * g + 2 * lane;   // k0 + 1 < Nk whenever k0 < Nk (Nk even)
                v[u][0] = v[u][1] = make_float2(0.f, 0.f);
                if (l < a.L && k0 < Nk) load_echo2<DT>(a.echo, ((long long)l * Nk + k0) >> 1, scale, v[u][0], v[u][1]);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 64 * g + 32 * h + lane;
                    v[u][h] = (l < a.L && k < Nk) ? load_echo<DT>(a.echo, (long long)l * Nk + k, scale)
                                                  : make_float2(0.f, 0.f);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kCompUnroll; ++u) {
            const int l = g0 + u;
            if (l >= a.L) continue;
            if (VEC) {
                const int k0 = 64 * g + 2 * lane;
                float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k0 < Nk) {
                    bad |= !(isfinite(v[u][0].x) && isfinite(v[u][0].y) && isfinite(v[u][1].x) && isfinite(v[u][1].y));
                    const uint32_t t0 = ph[u].x + (uint32_t)k0 * ph[u].y;   // exact mod 2^32
                    const float2 o0 = rotate_turns(v[u][0], t0), o1 = rotate_turns(v[u][1], t0 + ph[u].y);
                    out = make_float4(o0.x, o0.y, o1.x, o1.y);
                }
                __stcs(reinterpret_cast<float4 *>(a.shat) + ((long long)g * a.L + l) * kKC + lane, out);
            } else {
                float2 *dst = a.shat + ((long long)g * a.L + l) * (2 * kKC) + lane;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 64 * g + 32 * h + lane;
                    float2 out = make_float2(0.f, 0.f);
                    if (k < Nk) {
                        bad |= !(isfinite(v[u][h].x) && isfinite(v[u][h].y));
                        out = rotate_turns(v[u][h], ph[u].x + (uint32_t)k * ph[u].y);   // exact mod 2^32
                    }
                    __stcs(dst + 32 * h, out);
                }
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonfinite);
}

// Split output (tensor-core gridding): one warp per group of kCompUnroll
// samples and all their frequencies, in two passes.  Pass 1 bounds each
// sample's |s| over all frequencies by sqrt(2) max(|Re s|, |Im s|) (the
// rotation of Eq. 11 keeps |s|, so the echo gives it; every component of
// s_hat is at most that); the sample's exponent a puts the bound in
// [2^13, 2^14).  Pass 2 rotates (Eq. 11),
// scales by 2^a (exact) and stores every 64-frequency group as FP16 hi / lo
// planes: s_hat[g][l] = (hi[128 halves], lo[128 halves]).  The exponents
// go to sexp[l]; aref (one int) receives the max of 127 - a.  The second
// pass re-reads the warp's echo rows, which the first pass left in cache.
// One pass for scans of at most kSplitRegGroups frequency groups (Nk <= 256):
// U samples at a time, the lane's echo values of every group held in
// registers while the warp finds each sample's bound, then rotated, scaled
// and stored (the arithmetic of the two-pass form below, the same bits).
constexpr int kSplitRegGroups = 4, kSplitRegU = 2;

template <int DT, bool VEC>
__device__ __forceinline__ void compensate_split_regs(const PrepTailArgs &a, int g0, int n_g, float scale, bool &bad,
                                                      int &amax) {
    constexpr int U = kSplitRegU;
    const int lane = threadIdx.x & 31;
    const int Nk = a.Nk;
#pragma unroll 1
    for (int u0 = 0; u0 < kCompUnroll; u0 += U) {
        uint2 ph[U];
        float mc[U];
        float2 v[U][kSplitRegGroups][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int l = g0 + u0 + u;
            ph[u] = l < a.L ? __ldg(a.phase + l) : make_uint2(0u, 0u);
            mc[u] = 0.f;
#pragma unroll
            for (int g = 0; g < kSplitRegGroups; ++g) {
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (g < n_g && l < a.L) {
                    if (VEC) {
                        const int k0 = 64 * g + 2 * lane;
                        if (k0 < Nk) load_echo2<DT>(a.echo, ((long long)l * Nk + k0) >> 1, scale, v0, v1);
                    } else {
                        const int k = 64 * g + lane;
                        if (k < Nk) v0 = load_echo<DT>(a.echo, (long long)l * Nk + k, scale);
                        if (k + 32 < Nk) v1 = load_echo<DT>(a.echo, (long long)l * Nk + k + 32, scale);
                    }
                }
                v[u][g][0] = v0;
                v[u][g][1] = v1;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int g = 0; g < kSplitRegGroups; ++g)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 t = v[u][g][h];
                    bad |= !(isfinite(t.x) && isfinite(t.y));
                    mc[u] = fmaxf(mc[u], fmaxf(fabsf(t.x), fabsf(t.y)));
                }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) mc[u] = fmaxf(mc[u], __shfl_xor_sync(0xffffffffu, mc[u], off));
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int l = g0 + u0 + u;
            // every component of s_hat is at most |s| <= sqrt(2) max(|Re s|, |Im s|)
            const int ex = norm_exponent(mc[u] * 1.4142144f);
            const float sc = ldexpf(1.0f, ex);
            if (l >= a.L) continue;
            amax = max(amax, 127 - ex);
#pragma unroll
            for (int g = 0; g < kSplitRegGroups; ++g) {
                if (g >= n_g) continue;
                float2 o0 = make_float2(0.f, 0.f), o1 = o0;
                if (VEC) {
                    const int k0 = 64 * g + 2 * lane;
                    if (k0 < Nk) {
                        const uint32_t t0 = ph[u].x + (uint32_t)k0 * ph[u].y;   // exact mod 2^32
                        o0 = rotate_turns(v[u][g][0], t0);
                        o1 = rotate_turns(v[u][g][1], t0 + ph[u].y);
                    }
                } else {
                    const int k = 64 * g + lane;
                    if (k < Nk) o0 = rotate_turns(v[u][g][0], ph[u].x + (uint32_t)k * ph[u].y);
                    if (k + 32 < Nk) o1 = rotate_turns(v[u][g][1], ph[u].x + (uint32_t)(k + 32) * ph[u].y);
                }
                __half2 h0, l0, h1, l1;
                split2(o0.x, o0.y, sc, h0, l0);
                split2(o1.x, o1.y, sc, h1, l1);
                __half2 *row = reinterpret_cast<__half2 *>(a.shat) + ((long long)g * a.L + l) * 128;   // 512 B
                if (VEC) {   // complex 2 lane, 2 lane + 1 -> halves 4 lane .. 4 lane + 3
                    row[2 * lane] = h0;
                    row[2 * lane + 1] = h1;
                    row[64 + 2 * lane] = l0;
                    row[64 + 2 * lane + 1] = l1;
                } else {     // complex lane and 32 + lane
                    row[lane] = h0;
                    row[32 + lane] = h1;
                    row[64 + lane] = l0;
                    row[64 + 32 + lane] = l1;
                }
            }
            if (lane == 0) a.sexp[l] = (signed char)ex;
        }
    }
}

template <int DT, bool VEC>
__device__ __forceinline__ void compensate_split_body(const PrepTailArgs &a, int cblk) {
    __shared__ int amax_s[kPrepWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Nk = a.Nk, n_g = (((Nk + 31) >> 5) + 1) >> 1;
    const int warps = a.chunk_blocks * kPrepWarps;
    const float scale = (DT == MMSAR_ECHO_C64) ? 1.0f : *a.scale;
    bool bad = false;
    int amax = 0;
    for (int g0 = (cblk * kPrepWarps + warp) * kCompUnroll; g0 < a.L; g0 += warps * kCompUnroll) {
        if (n_g <= kSplitRegGroups) {   // one pass, the echo values kept in registers
            compensate_split_regs<DT, VEC>(a, g0, n_g, scale, bad, amax);
            continue;
        }
        uint2 ph[kCompUnroll];
        float mc[kCompUnroll];   // largest |Re s|, |Im s| of each sample (this lane's frequencies, then the warp's)
#pragma unroll
        for (int u = 0; u < kCompUnroll; ++u) {
            const int l = g0 + u;
            ph[u] = l < a.L ? __ldg(a.phase + l) : make_uint2(0u, 0u);
            mc[u] = 0.f;
        }
        // pass 1
        for (int g = 0; g < n_g; ++g) {
#pragma unroll
            for (int u = 0; u < kCompUnroll; ++u) {
                const int l = g0 + u;
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (VEC) {
                    const int k0 = 64 * g + 2 * lane;
                    if (l < a.L && k0 < Nk) load_echo2<DT>(a.echo, ((long long)l * Nk + k0) >> 1, scale, v0, v1);
                } else {
                    const int k = 64 * g + lane;
                    if (l < a.L && k < Nk) v0 = load_echo<DT>(a.echo, (long long)l * Nk + k, scale);
                    if (l < a.L && k + 32 < Nk) v1 = load_echo<DT>(a.echo, (long long)l * Nk + k + 32, scale);
                }
                bad |= !(isfinite(v0.x) && isfinite(v0.y) && isfinite(v1.x) && isfinite(v1.y));
                mc[u] = fmaxf(mc[u], fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v1.x), fabsf(v1.y))));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int u = 0; u < kCompUnroll; ++u) mc[u] = fmaxf(mc[u], __shfl_xor_sync(0xffffffffu, mc[u], off));
        int ex[kCompUnroll];
        float sc[kCompUnroll];
#pragma unroll
        for (int u = 0; u < kCompUnroll; ++u) {
            // every component of s_hat is at most |s| <= sqrt(2) max(|Re s|, |Im s|)
            // (bound rounded up; no squares, so no overflow)
            ex[u] = norm_exponent(mc[u] * 1.4142144f);
            sc[u] = ldexpf(1.0f, ex[u]);
            if (g0 + u < a.L) amax = max(amax, 127 - ex[u]);
        }
        // pass 2
        for (int g = 0; g < n_g; ++g) {
#pragma unroll
            for (int u = 0; u < kCompUnroll; ++u) {
                const int l = g0 + u;
                if (l >= a.L) continue;
                float2 o0 = make_float2(0.f, 0.f), o1 = o0;
                if (VEC) {
                    const int k0 = 64 * g + 2 * lane;
                    if (k0 < Nk) {
                        float2 v0, v1;
                        load_echo2<DT>(a.echo, ((long long)l * Nk + k0) >> 1, scale, v0, v1);
                        const uint32_t t0 = ph[u].x + (uint32_t)k0 * ph[u].y;   // exact mod 2^32
                        o0 = rotate_turns(v0, t0);
                        o1 = rotate_turns(v1, t0 + ph[u].y);
                    }
                } else {
                    const int k = 64 * g + lane;
                    if (k < Nk) o0 = rotate_turns(load_echo<DT>(a.echo, (long long)l * Nk + k, scale),
                                                  ph[u].x + (uint32_t)k * ph[u].y);
                    if (k + 32 < Nk) o1 = rotate_turns(load_echo<DT>(a.echo, (long long)l * Nk + k + 32, scale),
                                                       ph[u].x + (uint32_t)(k + 32) * ph[u].y);
                }
                __half2 h0, l0, h1, l1;
                split2(o0.x, o0.y, sc[u], h0, l0);
                split2(o1.x, o1.y, sc[u], h1, l1);
                __half2 *row = reinterpret_cast<__half2 *>(a.shat) + ((long long)g * a.L + l) * 128;   // 512 B
                if (VEC) {   // complex 2 lane, 2 lane + 1 -> halves 4 lane .. 4 lane + 3
                    row[2 * lane] = h0;
                    row[2 * lane + 1] = h1;
                    row[64 + 2 * lane] = l0;
                    row[64 + 2 * lane + 1] = l1;
                } else {     // complex lane and 32 + lane
                    row[lane] = h0;
                    row[32 + lane] = h1;
                    row[64 + lane] = l0;
                    row[64 + 32 + lane] = l1;
                }
            }
        }
        if (lane < kCompUnroll && g0 + lane < a.L) a.sexp[g0 + lane] = (signed char)ex[lane];
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonfinite);
    if (lane == 0) amax_s[warp] = amax;   // the reference exponent: one atomic per block
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int i = 0; i < kPrepWarps; ++i) m = max(m, amax_s[i]);
        if (m > 0) atomicMax(a.aref, m);
    }
}

template <int DT, bool VEC, bool SPLIT>
__global__ void __launch_bounds__(kPrepWarps * 32) compensate_kernel(const __grid_constant__ PrepTailArgs a) {
    compensate_body<DT, VEC, SPLIT>(a, blockIdx.x);
}

template <int DT, bool VEC, bool SPLIT>
__global__ void __launch_bounds__(kPrepWarps * 32)
    compensate_multi(const __grid_constant__ BatchTable<PrepTailArgs> t) {
    __shared__ PrepTailArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    compensate_body<DT, VEC, SPLIT>(sa, bid);
}

// the kernel instance: 2 x echo dtype + paired loads
static int compensate_describe(const Plan &p, void *ws, const void *echo, const float *scale, PrepTailArgs &a,
                               int &key) {
    char *w = reinterpret_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(w);
    a.n_bins = (int)p.n_bins;
    a.n_sort_blocks = (int)((p.n_bins + kPrepWarps - 1) / kPrepWarps);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.perm = reinterpret_cast<int *>(w + p.off_perm);
    a.rec = reinterpret_cast<const SampleRec *>(w + p.off_rec);
    a.w = p.w;
    a.kappa = (float)(1.5 * kPi / p.w);
    a.dd = reinterpret_cast<int2 *>(w + p.off_dd);
    a.wrec = reinterpret_cast<float4 *>(w + p.off_wq);
    a.tc = p.tc ? 1 : 0;
    a.trec = reinterpret_cast<int4 *>(w + p.off_trec);
    a.sexp = reinterpret_cast<signed char *>(w + p.off_sexp);
    a.aref = reinterpret_cast<int *>(w + p.off_aref);
    a.grouped = (p.grouped && !p.tc) ? 1 : 0;
    a.n_yrec_blocks = a.grouped ? (int)((p.L * (p.w + 4) + kPrepWarps * 32 - 1) / (kPrepWarps * 32)) : 0;
    a.P = p.shape.n_pos;
    a.R = p.shape.n_rx;
    a.TR = p.shape.n_tx * p.shape.n_rx;
    a.mry = p.mry;
    a.goff = reinterpret_cast<int4 *>(w + p.off_goff);
    a.grec = reinterpret_cast<const GroupRec *>(w + p.off_grec);
    a.cls = reinterpret_cast<const int *>(w + p.off_cls);
    a.gdd = reinterpret_cast<int2 *>(w + p.off_gdd);
    a.gxq = reinterpret_cast<float4 *>(w + p.off_gxq);
    a.yq = reinterpret_cast<float4 *>(w + p.off_yq);
    a.echo = echo;
    a.scale = scale;
    a.phase = reinterpret_cast<const uint2 *>(w + p.off_phase);
    a.Nk = p.shape.n_k;
    a.L = (int)p.L;
    const long long warps_needed = (p.L + kCompUnroll - 1) / kCompUnroll;
    long long cb = (warps_needed + kPrepWarps - 1) / kPrepWarps;
    if (cb > 152 * 32) cb = 152 * 32;
    a.chunk_blocks = (int)cb;
    a.err = &hdr->error;
    a.shat = reinterpret_cast<float2 *>(w + p.off_shat);
    // paired loads need an even Nk and an echo aligned to one pair
    const size_t pair_bytes = p.shape.dtype == MMSAR_ECHO_C64 ? 16 : 8;
    const bool vec = p.shape.n_k % 2 == 0 && reinterpret_cast<uintptr_t>(echo) % pair_bytes == 0;
    key = 8 * (p.tc ? 1 : 0) + 2 * (int)p.shape.dtype + (vec ? 1 : 0);
    // the split output covers every frequency group per warp (one exponent
    // per sample); the complex64 output runs one block range per group
    return (int)(a.n_sort_blocks + a.n_yrec_blocks + cb * (p.tc ? 1 : (p.n_kc + 1) / 2));
}

template <int DT, bool VEC, bool SPLIT>
static void compensate_launch(const PrepTailArgs *a, const BatchTable<PrepTailArgs> *t, int blocks, cudaStream_t s) {
    if (a)
        compensate_kernel<DT, VEC, SPLIT><<<blocks, kPrepWarps * 32, 0, s>>>(*a);
    else
        compensate_multi<DT, VEC, SPLIT><<<blocks, kPrepWarps * 32, 0, s>>>(*t);
}

template <bool SPLIT>
static void compensate_dispatch_dt(int key, const PrepTailArgs *a, const BatchTable<PrepTailArgs> *t, int blocks,
                                   cudaStream_t s) {
    switch (key & 7) {
        case 2 * MMSAR_ECHO_C64 + 1: compensate_launch<MMSAR_ECHO_C64, true, SPLIT>(a, t, blocks, s); break;
        case 2 * MMSAR_ECHO_C64: compensate_launch<MMSAR_ECHO_C64, false, SPLIT>(a, t, blocks, s); break;
        case 2 * MMSAR_ECHO_F16X2_SCALED + 1:
            compensate_launch<MMSAR_ECHO_F16X2_SCALED, true, SPLIT>(a, t, blocks, s);
            break;
        case 2 * MMSAR_ECHO_F16X2_SCALED:
            compensate_launch<MMSAR_ECHO_F16X2_SCALED, false, SPLIT>(a, t, blocks, s);
            break;
        case 2 * MMSAR_ECHO_BF16X2_SCALED + 1:
            compensate_launch<MMSAR_ECHO_BF16X2_SCALED, true, SPLIT>(a, t, blocks, s);
            break;
        default: compensate_launch<MMSAR_ECHO_BF16X2_SCALED, false, SPLIT>(a, t, blocks, s); break;
    }
}

// key: 8 x split output (tensor-core gridding) + 2 x echo dtype + paired loads
static void compensate_dispatch(int key, const PrepTailArgs *a, const BatchTable<PrepTailArgs> *t, int blocks,
                                cudaStream_t s) {
    if (key & 8)
        compensate_dispatch_dt<true>(key, a, t, blocks, s);
    else
        compensate_dispatch_dt<false>(key, a, t, blocks, s);
}

cudaError_t launch_compensate(const Plan &p, void *ws, const void *echo, const float *scale, cudaStream_t s) {
    PrepTailArgs a;
    int key;
    const int blocks = compensate_describe(p, ws, echo, scale, a, key);
    compensate_dispatch(key, &a, nullptr, blocks, s);
    return cudaGetLastError();
}

cudaError_t launch_compensate_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<PrepTailArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n);
    for (int i = 0; i < n; ++i)
        blocks[i] = compensate_describe(r[i].plan->p, r[i].workspace, r[i].echo, r[i].echo_scale, args[i], keys[i]);
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int key, const BatchTable<PrepTailArgs> &t, int total) {
                             compensate_dispatch(key, nullptr, &t, total, s);
                             return cudaGetLastError();
                         });
}

}  // namespace mmsar
