// Gaussian gridding (the spreading step of the fast Gaussian gridding NUFFT
// that Sec. III uses for FT_2D of Eq. 16) of the compensated virtual-array
// samples onto the 2Mx x 2My periodic aperture grid, in gather form.
//
// Weight of a sample at grid position g for cell j: exp(-kappa (g - j)^2)
// with kappa = h^2 / (4 tau) = 1.5 pi / w for the Greengard-Lee tau and a
// cell size h = 2 pi / (2M); the sample reaches the w cells
// u0 .. u0 + w - 1, u0 = ceil(g - w/2) (indices modulo the grid size).
//
// spread_weights_kernel (once per sample, bin order): the sample's offset
// inside its 4x4-cell bin and, per axis, w + 3 "quads" -- quad q holds the
// weights of taps q-3 .. q (zero outside 0..w-1), i.e. exactly the four
// weights a 4-cell block needs when it starts q - 3 cells after u0.
//
// spread_kernel: a CTA owns a 16x8 tile of grid cells and one chunk of 32
// frequencies; each of its 8 warps owns a 4x4 block of cells and keeps the
// 16 complex accumulators of its lane's frequency in registers.  Warps work
// independently (no block barrier): a warp walks the bins whose samples can
// reach its block, tests 32 samples at a time (one lane each) for overlap with
// the block and appends the overlapping ones to a list in shared memory, then
// applies the list with the loads of the entry two ahead already in flight.  For a bin d
// bins before the block, the block starts 4 d - (in-bin offset) cells after
// the sample's first tap, which selects one weight quad per axis (two 16-byte
// broadcast loads).  No two warps write the same cell: no atomics, a fixed
// summation order.
#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

__global__ void __launch_bounds__(256) spread_weights_kernel(const SampleRec *__restrict__ srec,
                                                             const WsHeader *__restrict__ hdr, int w, float kappa,
                                                             int *__restrict__ dd, float4 *__restrict__ wrec) {
    // one thread per record entry: consecutive threads write consecutive
    // 16-byte entries (entry 0 = header, then w + 3 x quads, w + 3 y quads)
    const int nq = w + 3, rq = 2 * nq + 1;
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = item / rq;
    if (s >= hdr->n_valid) return;
    const int e = (int)(item - s * rq);
    const SampleRec r = srec[s];
    if (e == 0) {
        const int d = (r.u0 & 3) | ((r.v0 & 3) << 2);
        dd[s] = d;
        wrec[item] = make_float4(__int_as_float(d), 0.f, 0.f, 0.f);
        return;
    }
    const int q = (e - 1) % nq;                   // quad q = taps q-3 .. q
    const float f = (e - 1) < nq ? r.fx : r.fy;
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int tap = q - 3 + i;
        const float d = f - (float)tap;
        v[i] = (tap >= 0 && tap < w) ? expf(-kappa * d * d) : 0.f;
    }
    wrec[item] = make_float4(v[0], v[1], v[2], v[3]);
}

cudaError_t launch_spread_weights(const Plan &p, void *ws, cudaStream_t s) {
    char *w = reinterpret_cast<char *>(ws);
    const long long items = p.L * (2 * (p.w + 3) + 1);
    const unsigned blocks = (unsigned)((items + 255) / 256);
    spread_weights_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const SampleRec *>(w + p.off_srec),
                                                 reinterpret_cast<const WsHeader *>(w), p.w,
                                                 (float)(1.5 * kPi / p.w), reinterpret_cast<int *>(w + p.off_dd),
                                                 reinterpret_cast<float4 *>(w + p.off_wq));
    return cudaGetLastError();
}

struct SpreadArgs {
    const float2 *shat;       // [n_kc][Lmax][32], bin order
    const int *dd;            // [Lmax] in-bin offsets du | dv << 2, bin order
    const float4 *wrec;       // [Lmax][2 (w + 3) + 1]: header + x quads + y quads
    const int *offsets;       // [n_bins + 1]
    float2 *G;                // [n_kc][mry][mrx][32]
    const WsHeader *hdr;      // occupied window of the grid
    long long Lmax;
    int mrx, mry, nbx, nby;
    int w, nb, n_kc;          // taps per axis; bins visited per axis; frequency chunks
};

// Does [t0, t0 + span) meet the periodic window lo .. lo + len - 1 (mod m)?
__device__ __forceinline__ bool tile_meets(int t0, int span, int lo, int len, int m) {
    if (len >= m) return true;
    if (len <= 0) return false;
    int d = (t0 - lo) % m;
    if (d < 0) d += m;
    int e = (lo - t0) % m;
    if (e < 0) e += m;
    return d < len || e < span;
}

constexpr int kSpreadThreads = 256;   // 8 warps: a 16 x 8-cell tile

constexpr int kListCap = 192;   // relevant samples listed per warp before they are applied

__global__ void __launch_bounds__(kSpreadThreads, 3) spread_kernel(SpreadArgs a) {
    // per warp: (x-quad index, y-quad index, sample index) of each listed sample
    __shared__ int4 lists[kSpreadThreads / 32][kListCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = a.mrx >> 4;
    // the frequency chunk varies fastest, so the chunks of one tile run
    // together and share the tile's weight records in L2
    const int kc = blockIdx.x % a.n_kc;
    const int tile = blockIdx.x / a.n_kc;
    // tiles outside the occupied window stay unwritten: the FFT along x'
    // reads only the window and takes the rest as zero
    if (!tile_meets((tile % tiles_x) * 16, 16, a.hdr->u_lo, a.hdr->u_len, a.mrx) ||
        !tile_meets((tile / tiles_x) * 8, 8, a.hdr->v_lo, a.hdr->v_len, a.mry))
        return;
    const int U = (tile % tiles_x) * 16 + (warp & 3) * 4;
    const int V = (tile / tiles_x) * 8 + (warp >> 2) * 4;
    const int rq = 2 * (a.w + 3) + 1;
    const int nq = a.w + 3;
    float2 acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = make_float2(0.f, 0.f);
    const float2 *sh = a.shat + (long long)kc * a.Lmax * kKC + lane;
    int4 *list = lists[warp];

    // apply the listed samples through a three-deep pipeline: the loads of
    // entry i + 3 are issued as soon as entry i has been accumulated
    auto apply = [&](int n) {
        float4 x0, y0, x1, y1, x2, y2;
        float2 v0, v1, v2;
        auto fetch = [&](int i, float4 &x, float4 &y, float2 &v) {
            const int4 e = list[i];
            x = __ldg(a.wrec + e.x);
            y = __ldg(a.wrec + e.y);
            v = __ldg(sh + (e.z << 5));
        };
        auto consume = [&](const float4 &x, const float4 &y, const float2 &v) {
            const float wx[4] = {x.x, x.y, x.z, x.w};
            const float wy[4] = {y.x, y.y, y.z, y.w};
            // (re, im) pairs in packed two-lane FP32 instructions
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 t = fmul2(make_float2(wy[j], wy[j]), v);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[j][i] = ffma2(make_float2(wx[i], wx[i]), t, acc[j][i]);
            }
        };
        if (n > 0) fetch(0, x0, y0, v0);
        if (n > 1) fetch(1, x1, y1, v1);
        if (n > 2) fetch(2, x2, y2, v2);
        for (int i = 0; i < n; i += 3) {
            consume(x0, y0, v0);
            if (i + 3 < n) fetch(i + 3, x0, y0, v0);
            if (i + 1 >= n) break;
            consume(x1, y1, v1);
            if (i + 4 < n) fetch(i + 4, x1, y1, v1);
            if (i + 2 >= n) break;
            consume(x2, y2, v2);
            if (i + 5 < n) fetch(i + 5, x2, y2, v2);
        }
    };

    const int bu0 = U >> 2, bv0 = V >> 2;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int dbv = a.nb - 1; dbv >= 0; --dbv) {
        int bv = bv0 - dbv;
        if (bv < 0) bv += a.nby;
        for (int dbu = a.nb - 1; dbu >= 0; --dbu) {
            int bu = bu0 - dbu;
            if (bu < 0) bu += a.nbx;
            const int bin = bv * a.nbx + bu;
            const int beg = __ldg(a.offsets + bin), end = __ldg(a.offsets + bin + 1);
            for (int s0 = beg; s0 < end; s0 += 32) {
                // which of the next 32 samples reach this block, in one step
                const int my = s0 + lane;
                bool rel = false;
                int4 ent = make_int4(0, 0, 0, 0);
                if (my < end) {
                    const int d = __ldg(a.dd + my);
                    const int ru = 4 * dbu - (d & 3);     // block start relative to the first tap, >= -3
                    const int rv = 4 * dbv - (d >> 2);
                    rel = ru < a.w && rv < a.w;
                    const int base = my * rq + 1;         // the sample's x quads, then its y quads
                    ent = make_int4(base + ru + 3, base + nq + rv + 3, my, 0);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, rel);
                if (n + __popc(mask) > kListCap) {   // keep the list within its buffer
                    __syncwarp();
                    apply(n);
                    n = 0;
                    __syncwarp();
                }
                if (rel) list[n + __popc(mask & lt)] = ent;
                n += __popc(mask);
            }
        }
    }
    __syncwarp();
    apply(n);
    float2 *g = a.G + (long long)kc * a.mry * a.mrx * kKC;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) g[((long long)(V + j) * a.mrx + (U + i)) * kKC + lane] = acc[j][i];
}

cudaError_t launch_spread(const Plan &p, void *ws, cudaStream_t s) {
    char *w = reinterpret_cast<char *>(ws);
    SpreadArgs a;
    a.shat = reinterpret_cast<const float2 *>(w + p.off_shat);
    a.dd = reinterpret_cast<const int *>(w + p.off_dd);
    a.wrec = reinterpret_cast<const float4 *>(w + p.off_wq);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.G = reinterpret_cast<float2 *>(w + p.off_G);
    a.hdr = reinterpret_cast<const WsHeader *>(w);
    a.Lmax = p.L;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.nby = p.nby;
    a.w = p.w;
    a.nb = (p.w - 1 + kBin - 1) / kBin + 1;
    a.n_kc = p.n_kc;
    const unsigned blocks = (unsigned)((p.mrx / 16) * (p.mry / 8) * p.n_kc);
    spread_kernel<<<blocks, kSpreadThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mmsar
