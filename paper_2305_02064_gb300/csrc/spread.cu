// Gaussian gridding (the spreading step of the fast Gaussian gridding NUFFT
// that Sec. III uses for FT_2D of Eq. 16) of the compensated virtual-array
// samples onto the 2Mx x 2My periodic aperture grid, in gather form.
//
// Work decomposition: a CTA owns a 16x16 tile of grid cells and one chunk of
// 32 frequencies; each of its 16 warps owns a 4x4 block of cells and keeps the
// 16 complex accumulators of its lane's frequency in registers.  A warp visits
// only the bins (4x4 cells each, samples sorted by bin) whose samples can
// reach its block, so no two warps ever write the same cell and no atomics
// are used.  The Gaussian weights depend on the sample only, so each lane
// applies the same 8 weights (4 per axis) to its own frequency.
//
// Weight of a sample at grid position g for cell j: exp(-kappa (g - j)^2)
// with kappa = h^2 / (4 tau) = 1.5 pi / w for the Greengard-Lee tau and a
// cell size h = 2 pi / (2M); the sample reaches the w cells
// ceil(g - w/2) .. ceil(g - w/2) + w - 1 (indices modulo the grid size).
#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

struct SpreadArgs {
    const float2 *shat;       // [n_kc][Lmax][32], bin order
    const SampleRec *srec;    // [Lmax], bin order
    const int *offsets;       // [n_bins + 1]
    float2 *G;                // [n_kc][mry][mrx][32]
    long long Lmax;
    int mrx, mry, nbx, nby;
    int w, nb;                // taps per axis; bins visited per axis
    float kappa;
};

__global__ void __launch_bounds__(512, 2) spread_kernel(SpreadArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = a.mrx >> 4;
    const int kc = blockIdx.y;
    const int U = (blockIdx.x % tiles_x) * 16 + (warp & 3) * 4;
    const int V = (blockIdx.x / tiles_x) * 16 + (warp >> 2) * 4;
    const int half_x = a.mrx >> 1, half_y = a.mry >> 1;
    float2 acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = make_float2(0.f, 0.f);
    const float2 *sh = a.shat + (long long)kc * a.Lmax * kKC + lane;
    const int bu0 = U >> 2, bv0 = V >> 2;
    for (int dbv = a.nb - 1; dbv >= 0; --dbv) {
        int bv = bv0 - dbv;
        if (bv < 0) bv += a.nby;
        for (int dbu = a.nb - 1; dbu >= 0; --dbu) {
            int bu = bu0 - dbu;
            if (bu < 0) bu += a.nbx;
            const int bin = bv * a.nbx + bu;
            const int beg = __ldg(a.offsets + bin), end = __ldg(a.offsets + bin + 1);
            for (int s = beg; s < end; ++s) {
                const SampleRec r = a.srec[s];
                int ru = U - r.u0;
                if (ru > half_x) ru -= a.mrx; else if (ru <= -half_x) ru += a.mrx;
                int rv = V - r.v0;
                if (rv > half_y) rv -= a.mry; else if (rv <= -half_y) rv += a.mry;
                if (ru < -3 || ru >= a.w || rv < -3 || rv >= a.w) continue;
                float wx[4], wy[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ta = ru + i, tb = rv + i;
                    const float dxa = r.fx - (float)ta, dyb = r.fy - (float)tb;
                    wx[i] = (ta >= 0 && ta < a.w) ? __expf(-a.kappa * dxa * dxa) : 0.f;
                    wy[i] = (tb >= 0 && tb < a.w) ? __expf(-a.kappa * dyb * dyb) : 0.f;
                }
                const float2 v = __ldg(sh + (long long)s * kKC);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 t = make_float2(wy[j] * v.x, wy[j] * v.y);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[j][i].x = fmaf(wx[i], t.x, acc[j][i].x);
                        acc[j][i].y = fmaf(wx[i], t.y, acc[j][i].y);
                    }
                }
            }
        }
    }
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
    a.srec = reinterpret_cast<const SampleRec *>(w + p.off_srec);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.G = reinterpret_cast<float2 *>(w + p.off_G);
    a.Lmax = p.L;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.nby = p.nby;
    a.w = p.w;
    a.nb = (p.w - 1 + kBin - 1) / kBin + 1;
    a.kappa = (float)(1.5 * kPi / p.w);
    dim3 grid((unsigned)((p.mrx / 16) * (p.mry / 16)), p.n_kc);
    spread_kernel<<<grid, 512, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mmsar
