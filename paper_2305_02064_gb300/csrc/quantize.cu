// Reduced-precision echo storage: per-scan max-abs scaling of a complex64
// echo into interleaved FP16 or BF16 pairs.  (The paper stores echoes as
// MATLAB doubles; halving the echo bytes halves the compensation stage's
// compulsory reads, and the arithmetic stays FP32 after the load.)
//
// Pass 1: the largest |Re| or |Im| of the scan, reduced with warp shuffles
// per block and combined across blocks by an integer atomicMax on the float's
// bit pattern (order-preserving for non-negative floats, so the result does
// not depend on the order of the blocks).
// Pass 2: scale = max / 16384 (keeps FP16 values well inside its normal
// range), q = (s / scale) rounded to the storage type.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace mmsar {

constexpr float kQuantHeadroom = 16384.0f;

__global__ void __launch_bounds__(256) maxabs_kernel(const float4 *__restrict__ v4, long long n4,
                                                     const float *__restrict__ tail, int ntail, int *bits) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n4; i += (long long)gridDim.x * 256) {
        const float4 v = __ldg(v4 + i);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < ntail; i += 256) m = fmaxf(m, fabsf(tail[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < 8; ++w) b = fmaxf(b, wm[w]);
        if (!(b <= 3.0e38f)) b = 3.0e38f;   // NaN / Inf: saturate (reported by the imaging call)
        atomicMax(bits, __float_as_int(b));
    }
}

template <int DT>
__global__ void __launch_bounds__(256) quantize_kernel(const float2 *__restrict__ in, long long n,
                                                       const int *__restrict__ bits, float *__restrict__ scale_out,
                                                       void *__restrict__ out) {
    const float mx = __int_as_float(*bits);
    const float scale = mx > 0.f ? mx / kQuantHeadroom : 1.0f;
    const float inv = 1.0f / scale;
    if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = scale;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float2 v = __ldg(in + i);
        if (DT == MMSAR_ECHO_F16X2_SCALED)
            reinterpret_cast<__half2 *>(out)[i] = __floats2half2_rn(v.x * inv, v.y * inv);
        else
            reinterpret_cast<__nv_bfloat162 *>(out)[i] = __floats2bfloat162_rn(v.x * inv, v.y * inv);
    }
}

}  // namespace mmsar

using namespace mmsar;

extern "C" mmsar_status mmsar_quantize_echo(const void *echo_c64, int64_t n_complex, mmsar_echo_dtype dtype,
                                            void *out, float *scale, int *scratch, void *stream) {
    if (!echo_c64 || !out || !scale || !scratch || n_complex < 0)
        return report_error(MMSAR_ERR_INVALID_ARG, "bad argument to mmsar_quantize_echo");
    if (dtype != MMSAR_ECHO_F16X2_SCALED && dtype != MMSAR_ECHO_BF16X2_SCALED)
        return report_error(MMSAR_ERR_INVALID_ARG, "quantisation targets FP16 or BF16 pairs");
    if (reinterpret_cast<uintptr_t>(echo_c64) % 16 != 0)
        return report_error(MMSAR_ERR_INVALID_ARG, "echo must be 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int), s);
    if (e != cudaSuccess) return report_error(MMSAR_ERR_CUDA, "quantize: %s", cudaGetErrorString(e));
    if (n_complex == 0) return MMSAR_OK;
    const long long nf = 2 * n_complex;   // floats
    const long long n4 = nf / 4;
    const int ntail = (int)(nf - 4 * n4);
    const float *f = reinterpret_cast<const float *>(echo_c64);
    long long blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    maxabs_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(f), n4, f + 4 * n4, ntail,
                                                   scratch);
    long long qb = (n_complex + 255) / 256;
    if (qb > 152 * 16) qb = 152 * 16;
    if (dtype == MMSAR_ECHO_F16X2_SCALED)
        quantize_kernel<MMSAR_ECHO_F16X2_SCALED><<<(unsigned)qb, 256, 0, s>>>(
            reinterpret_cast<const float2 *>(echo_c64), n_complex, scratch, scale, out);
    else
        quantize_kernel<MMSAR_ECHO_BF16X2_SCALED><<<(unsigned)qb, 256, 0, s>>>(
            reinterpret_cast<const float2 *>(echo_c64), n_complex, scratch, scale, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? MMSAR_OK : report_error(MMSAR_ERR_CUDA, "quantize: %s", cudaGetErrorString(e));
}
