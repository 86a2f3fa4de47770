// Direct back-projection (the paper's gold-standard reference algorithm,
// Sec. III and Sec. V): for every voxel r
//     o_BP(r) = sum_{t, r, p, k} s(t, r, p, k) exp(+j k_k (|T_tp - r| + |R_rp - r|)),
// k_k = 2 pi (f0 + k df) / c (Eq. 2 round trip, Eq. 9 wavenumber), no
// normalisation.  It is a different operator from the RMA (no Eq. 7
// approximation, no k_z weight) and is used as an independent cross-check of
// image peaks; its cost is voxels x samples x frequencies.
//
// One thread per voxel; a CTA stages a few samples at a time (their Tx/Rx
// positions and echo rows) in shared memory and every thread sweeps them.
// Precision: the round trip and the phase arguments f0 R / c and df R / c
// are FP64 per (voxel, sample), reduced to 32-bit fixed-point turns; over k
// the phase rotates by a complex recurrence in FP32, re-anchored from the
// exact fixed-point phase every 32 frequencies.
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

constexpr int kBpaThreads = 256;
constexpr int kBpaStage = 8;   // samples per shared-memory stage

__device__ __forceinline__ uint32_t turns_fixed(double turns) {
    const double f = turns - floor(turns);
    return (uint32_t)(unsigned long long)llrint(f * 4294967296.0);
}

__device__ __forceinline__ float2 unit_from_fixed(uint32_t t) {
    float s, c;
    sincospif((float)(int32_t)t * 4.6566128730773926e-10f, &s, &c);   // angle 2 pi t / 2^32
    return make_float2(c, s);
}

struct BpaArgs {
    const float2 *echo;      // [T][R][P][Nk]
    const double *pos, *tx, *rx;
    const double *vox;       // [n][3] or null: the plan's grid
    long long n;
    int T, R, P, Nk;
    double x0, y0, z0, dx, dy, dz;
    int ny, nz;
    double f0_c, df_c;       // f0 / c, df / c
    float2 *out;
};

__global__ void __launch_bounds__(kBpaThreads) bpa_kernel(BpaArgs a) {
    extern __shared__ float2 sh_echo[];                 // [kBpaStage][Nk]
    __shared__ double sh_geo[kBpaStage][6];             // Tx xyz, Rx xyz
    const long long v = (long long)blockIdx.x * kBpaThreads + threadIdx.x;
    double X = 0, Y = 0, Z = 0;
    if (v < a.n) {
        if (a.vox) {
            X = a.vox[3 * v];
            Y = a.vox[3 * v + 1];
            Z = a.vox[3 * v + 2];
        } else {
            const long long i = v / ((long long)a.ny * a.nz);
            const long long rem = v - i * a.ny * a.nz;
            const long long j = rem / a.nz, q = rem - j * a.nz;
            X = a.x0 + i * a.dx;
            Y = a.y0 + j * a.dy;
            Z = a.z0 + q * a.dz;
        }
    }
    float2 acc = make_float2(0.f, 0.f);
    const long long L = (long long)a.T * a.R * a.P;
    for (long long l0 = 0; l0 < L; l0 += kBpaStage) {
        const int ns = (int)min((long long)kBpaStage, L - l0);
        __syncthreads();
        if (threadIdx.x < ns) {
            const long long l = l0 + threadIdx.x;
            const int p = (int)(l % a.P), r = (int)((l / a.P) % a.R), t = (int)(l / ((long long)a.P * a.R));
            for (int c = 0; c < 3; ++c) {
                sh_geo[threadIdx.x][c] = a.pos[3 * p + c] + a.tx[3 * t + c];
                sh_geo[threadIdx.x][3 + c] = a.pos[3 * p + c] + a.rx[3 * r + c];
            }
        }
        for (int e = threadIdx.x; e < ns * a.Nk; e += kBpaThreads)
            sh_echo[e] = __ldg(a.echo + l0 * a.Nk + e);
        __syncthreads();
        if (v >= a.n) continue;
        for (int s = 0; s < ns; ++s) {
            const double *g = sh_geo[s];
            const double ax = g[0] - X, ay = g[1] - Y, az = g[2] - Z;
            const double bx = g[3] - X, by = g[4] - Y, bz = g[5] - Z;
            const double Rrt = sqrt(ax * ax + ay * ay + az * az) + sqrt(bx * bx + by * by + bz * bz);
            const uint32_t ta = turns_fixed(a.f0_c * Rrt), tb = turns_fixed(a.df_c * Rrt);
            const float2 rho = unit_from_fixed(tb);
            const float2 *row = sh_echo + s * a.Nk;
            for (int k0 = 0; k0 < a.Nk; k0 += 32) {
                float2 z = unit_from_fixed(ta + (uint32_t)k0 * tb);   // exact anchor
                const int k1 = min(a.Nk, k0 + 32);
                for (int k = k0; k < k1; ++k) {
                    const float2 sk = row[k];
                    acc.x = fmaf(sk.x, z.x, fmaf(-sk.y, z.y, acc.x));
                    acc.y = fmaf(sk.x, z.y, fmaf(sk.y, z.x, acc.y));
                    z = cmul(z, rho);
                }
            }
        }
    }
    if (v < a.n) a.out[v] = acc;
}

}  // namespace mmsar

using namespace mmsar;

extern "C" mmsar_status mmsar_backproject(const mmsar_plan *plan, const void *echo, const double *pos,
                                          const double *tx, const double *rx, const double *voxels, int64_t n_voxels,
                                          void *out, void *stream) {
    if (!plan) return report_error(MMSAR_ERR_INVALID_ARG, "null plan");
    const Plan &p = plan->p;
    if (p.shape.dtype != MMSAR_ECHO_C64)
        return report_error(MMSAR_ERR_INVALID_ARG, "back-projection reads complex64 echoes");
    if (!out || (p.L > 0 && (!echo || !pos || !tx || !rx)))
        return report_error(MMSAR_ERR_INVALID_ARG, "null pointer to mmsar_backproject");
    const long long nv = voxels ? (long long)n_voxels : (long long)p.grid.nx * p.grid.ny * p.grid.nz;
    if (nv < 0) return report_error(MMSAR_ERR_INVALID_ARG, "negative voxel count");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nv == 0) return MMSAR_OK;
    BpaArgs a;
    a.echo = reinterpret_cast<const float2 *>(echo);
    a.pos = pos;
    a.tx = tx;
    a.rx = rx;
    a.vox = voxels;
    a.n = nv;
    a.T = p.shape.n_tx;
    a.R = p.shape.n_rx;
    a.P = p.shape.n_pos;
    a.Nk = p.shape.n_k;
    a.x0 = p.grid.x0;
    a.y0 = p.grid.y0;
    a.z0 = p.grid.z0;
    a.dx = p.grid.dx;
    a.dy = p.grid.dy;
    a.dz = p.grid.dz;
    a.ny = p.grid.ny;
    a.nz = p.grid.nz;
    a.f0_c = p.shape.f0_hz / kC0;
    a.df_c = p.shape.df_hz / kC0;
    a.out = reinterpret_cast<float2 *>(out);
    const size_t smem = (size_t)kBpaStage * p.shape.n_k * sizeof(float2);
    cudaError_t e = ensure_smem_attr((const void *)bpa_kernel, smem);
    if (e != cudaSuccess) return report_error(MMSAR_ERR_CUDA, "back-projection: %s", cudaGetErrorString(e));
    bpa_kernel<<<(unsigned)((nv + kBpaThreads - 1) / kBpaThreads), kBpaThreads, smem, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? MMSAR_OK : report_error(MMSAR_ERR_CUDA, "back-projection: %s", cudaGetErrorString(e));
}
