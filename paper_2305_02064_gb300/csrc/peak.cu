// Peak voxel of a complex volume: the largest |o| and the lowest linear index
// whose |o| is within 1e-6 (relative) of it.  Two grid-stride passes with
// warp-shuffle reductions; the block partials are combined by one block, so
// the result does not depend on scheduling.
#include "internal.cuh"

namespace mmsar {

constexpr int kPeakBlocks = 1024;
constexpr int kPeakThreads = 256;

struct PeakScratch {
    float block_max[kPeakBlocks];
    long long block_idx[kPeakBlocks];
    float max_abs;
};

__device__ __forceinline__ float cabs2(float2 v) { return sqrtf(v.x * v.x + v.y * v.y); }

__global__ void __launch_bounds__(kPeakThreads) peak_max_kernel(const float2 *__restrict__ vol, long long n,
                                                              PeakScratch *sc) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * kPeakThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kPeakThreads)
        m = fmaxf(m, cabs2(__ldg(vol + i)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[kPeakThreads / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < kPeakThreads / 32; ++w) b = fmaxf(b, wm[w]);
        sc->block_max[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(kPeakThreads) peak_combine_max(PeakScratch *sc, int nb) {
    float m = 0.f;
    for (int i = threadIdx.x; i < nb; i += kPeakThreads) m = fmaxf(m, sc->block_max[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[kPeakThreads / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < kPeakThreads / 32; ++w) b = fmaxf(b, wm[w]);
        sc->max_abs = b;
    }
}

__global__ void __launch_bounds__(kPeakThreads) peak_index_kernel(const float2 *__restrict__ vol, long long n,
                                                                PeakScratch *sc) {
    const float thr = sc->max_abs * (1.0f - 1e-6f);
    long long best = n;
    for (long long i = (long long)blockIdx.x * kPeakThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kPeakThreads) {
        if (cabs2(__ldg(vol + i)) >= thr) {
            best = i;
            break;   // indices only grow along this thread's stride
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ long long wb[kPeakThreads / 32];
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = n;
        for (int w = 0; w < kPeakThreads / 32; ++w) b = min(b, wb[w]);
        sc->block_idx[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(kPeakThreads) peak_finish(const PeakScratch *sc, int nb, long long n,
                                                          void *result) {
    long long b = n;
    for (int i = threadIdx.x; i < nb; i += kPeakThreads) b = min(b, sc->block_idx[i]);
    for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(0xffffffffu, b, o));
    __shared__ long long wb[kPeakThreads / 32];
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long r = n;
        for (int w = 0; w < kPeakThreads / 32; ++w) r = min(r, wb[w]);
        *reinterpret_cast<long long *>(result) = r < n ? r : 0;
        reinterpret_cast<float *>(result)[2] = sc->max_abs;
    }
}

size_t peak_scratch_bytes(int64_t) { return (sizeof(PeakScratch) + 255) / 256 * 256; }

cudaError_t launch_peak(const void *vol, int64_t n, void *scratch, void *result, cudaStream_t s) {
    const float2 *v = reinterpret_cast<const float2 *>(vol);
    PeakScratch *sc = reinterpret_cast<PeakScratch *>(scratch);
    long long nb = (n + kPeakThreads - 1) / kPeakThreads;
    if (nb > kPeakBlocks) nb = kPeakBlocks;
    peak_max_kernel<<<(unsigned)nb, kPeakThreads, 0, s>>>(v, n, sc);
    peak_combine_max<<<1, kPeakThreads, 0, s>>>(sc, (int)nb);
    peak_index_kernel<<<(unsigned)nb, kPeakThreads, 0, s>>>(v, n, sc);
    peak_finish<<<1, kPeakThreads, 0, s>>>(sc, (int)nb, n, result);
    return cudaGetLastError();
}

}  // namespace mmsar
