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
// One warp per column.  Because k_z grows with k, the samples of a column
// are already sorted along the gridding axis, so each lane gathers one grid
// point from the contiguous range of samples within reach (binary search)
// -- no atomics, a fixed summation order.  The FFT then runs over the
// 8 columns of the CTA in shared memory (fft.cuh).
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

struct StoltArgs {
    const float2 *S;        // [mx][my][nkp]
    float2 *Z;              // [mx][my][nz]
    const WsHeader *hdr;
    int mx, my, nk, nkp, nz, w;
    double kx_step, ky_step;   // 2 pi / (M d)
    double k0, dk;             // 2 pi f0 / c, 2 pi df / c
    double dz, z_c;
    float kappa;
    float deapod_scale;        // sqrt(pi / tau_z) / MRZ
    float tau_z;
};

constexpr int kStoltCols = 8;

template <int MRZ>
__global__ void __launch_bounds__(256) stolt_kernel(StoltArgs a) {
    extern __shared__ float2 smem[];
    float2 *grid = smem;                                  // [MRZ][8]
    float2 *tw = grid + MRZ * kStoltCols;                 // [MRZ]
    float2 *cbuf = tw + MRZ;                              // [8][nk]
    float *tbuf = reinterpret_cast<float *>(cbuf + kStoltCols * a.nk);  // [8][nk]
    float *kk = tbuf + kStoltCols * a.nk;                 // [nk]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncol = a.mx * a.my;
    const int col = blockIdx.x * kStoltCols + warp;
    for (int e = tid; e < MRZ * kStoltCols; e += 256) grid[e] = make_float2(0.f, 0.f);
    for (int k = tid; k < a.nk; k += 256) kk[k] = (float)(a.k0 + a.dk * k);
    fill_twiddles<MRZ, +1>(tw, tid, 256);
    __syncthreads();
    if (col < ncol) {
        float2 *cw = cbuf + warp * a.nk;
        float *tw_ = tbuf + warp * a.nk;
        const int om = col / a.my, on = col - (col / a.my) * a.my;
        const float kx = (float)((om - a.mx / 2) * a.kx_step);
        const float ky = (float)((on - a.my / 2) * a.ky_step);
        const float kr2 = kx * kx + ky * ky;
        const double zoff = a.z_c - a.hdr->z_ref;
        const float turns_per_kz = (float)(zoff / (2.0 * kPi));
        const float cells_per_kz = (float)(a.dz * MRZ / (2.0 * kPi));
        const float2 *Sc = a.S + (long long)col * a.nkp;
        int n_evan = 0;
        for (int k0 = 0; k0 < a.nk; k0 += 32) {
            const int k = k0 + lane;
            bool evan = false;
            if (k < a.nk) {
                const float kv = kk[k];
                const float kz2 = 4.f * kv * kv - kr2;
                float2 c = make_float2(0.f, 0.f);
                float t = -1e30f;
                if (kz2 > 0.f) {
                    const float kz = sqrtf(kz2);
                    t = kz * cells_per_kz;
                    float ph = kz * turns_per_kz;
                    ph -= rintf(ph);
                    float sn, cs;
                    sincospif(2.f * ph, &sn, &cs);
                    const float2 s = __ldg(Sc + k);
                    c = cmul(make_float2(s.x * kz, s.y * kz), make_float2(cs, sn));
                } else {
                    evan = true;
                }
                cw[k] = c;
                tw_[k] = t;
            }
            n_evan += __popc(__ballot_sync(0xffffffffu, evan));
        }
        __syncwarp();
        const int kf = n_evan;   // k_z increases with k: evanescent samples form a prefix
        if (kf < a.nk) {
            const float hw = 0.5f * a.w;
            const int jlo = (int)ceilf(tw_[kf] - hw);
            const int jhi = (int)ceilf(tw_[a.nk - 1] - hw) + a.w - 1;
            for (int jb = jlo; jb <= jhi; jb += 32) {
                const int j = jb + lane;
                if (j <= jhi) {
                    const float lo_t = (float)j - hw, hi_t = (float)j + hw;
                    // first sample with t > lo_t
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
                    float2 &gref = grid[(j & (MRZ - 1)) * kStoltCols + warp];
                    gref = cadd(gref, acc);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    smem_fft<MRZ, kStoltCols, 256, +1>(grid, tw);
    if (col < ncol) {
        float2 *Zc = a.Z + (long long)col * a.nz;
        for (int q = lane; q < a.nz; q += 32) {
            const int qp = q - a.nz / 2;
            const float sc = a.deapod_scale * __expf((float)(qp * qp) * a.tau_z);
            const float2 v = grid[(qp & (MRZ - 1)) * kStoltCols + warp];
            Zc[q] = make_float2(v.x * sc, v.y * sc);
        }
    }
}

template <int MRZ>
static cudaError_t launch_mrz(const StoltArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)(MRZ * kStoltCols + MRZ) * sizeof(float2) +
                        (size_t)kStoltCols * a.nk * (sizeof(float2) + sizeof(float)) + (size_t)a.nk * sizeof(float);
    cudaError_t e = ensure_smem_attr((const void *)stolt_kernel<MRZ>, smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((a.mx * a.my + kStoltCols - 1) / kStoltCols);
    stolt_kernel<MRZ><<<blocks, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stolt(const Plan &p, void *ws, cudaStream_t s) {
    char *w = reinterpret_cast<char *>(ws);
    StoltArgs a;
    a.S = reinterpret_cast<const float2 *>(w + p.off_S);
    a.Z = reinterpret_cast<float2 *>(w + p.off_Z);
    a.hdr = reinterpret_cast<const WsHeader *>(w);
    a.mx = p.mx;
    a.my = p.my;
    a.nk = p.shape.n_k;
    a.nkp = p.nkp;
    a.nz = p.grid.nz;
    a.w = p.w;
    a.kx_step = 2.0 * kPi / (p.mx * p.grid.dx);
    a.ky_step = 2.0 * kPi / (p.my * p.grid.dy);
    a.k0 = 2.0 * kPi * p.shape.f0_hz / kC0;
    a.dk = 2.0 * kPi * p.shape.df_hz / kC0;
    a.dz = p.grid.dz;
    a.z_c = p.grid.z0 + (p.grid.nz / 2) * p.grid.dz;
    a.kappa = (float)(1.5 * kPi / p.w);
    a.deapod_scale = (float)(std::sqrt(kPi / p.tau_z) / p.mrz);
    a.tau_z = (float)p.tau_z;
    switch (p.mrz) {
        case 32: return launch_mrz<32>(a, s);
        case 64: return launch_mrz<64>(a, s);
        case 128: return launch_mrz<128>(a, s);
        case 256: return launch_mrz<256>(a, s);
        case 512: return launch_mrz<512>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mmsar
