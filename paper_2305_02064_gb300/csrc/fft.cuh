// Shared-memory Stockham FFT along the row axis of a [L][P] tile (C columns,
// row pitch P).
//
// The tile holds C independent columns (contiguous in shared memory, so a
// warp's lanes touch consecutive 8-byte words and the accesses are
// conflict-free); every column is transformed along its L rows.  Passes are
// radix 8 or 4, chosen so that L = 4^a 8^b; each pass loads its R inputs
// into registers, applies the twiddles, runs an R-point DFT and stores the
// outputs in self-sorting (Stockham) order, so the result is in natural
// order after the last pass.  SIGN = -1 is the forward transform
// sum_n x_n exp(-2 pi i k n / L), SIGN = +1 the unnormalised inverse.
#pragma once

#include <cuda_runtime.h>

namespace mmsar {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Packed two-lane FP32 operations of sm_100-family tensor-less ALUs
// (fma/mul.rn.f32x2): each lane is rounded exactly like the scalar
// instruction, one instruction does both.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {   // a * b + c
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by SIGN * i
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = fadd2(a0, a2), t1 = fsub2(a0, a2);
    const float2 t2 = fadd2(a1, a3), t3 = mul_si<SIGN>(fsub2(a1, a3));
    a0 = fadd2(t0, t2);
    a2 = fsub2(t0, t2);
    a1 = fadd2(t1, t3);
    a3 = fsub2(t1, t3);
}

template <int SIGN>
__device__ __forceinline__ void dft8(float2 *v) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    const float r = 0.70710678118654752440f;
    // o_k *= exp(SIGN * 2 pi i k / 8)
    o1 = make_float2(r * (o1.x - SIGN * o1.y), r * (o1.y + SIGN * o1.x));
    o2 = mul_si<SIGN>(o2);
    o3 = make_float2(r * (-o3.x - SIGN * o3.y), r * (-o3.y + SIGN * o3.x));
    v[0] = fadd2(e0, o0); v[4] = fsub2(e0, o0);
    v[1] = fadd2(e1, o1); v[5] = fsub2(e1, o1);
    v[2] = fadd2(e2, o2); v[6] = fsub2(e2, o2);
    v[3] = fadd2(e3, o3); v[7] = fsub2(e3, o3);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2 *v) {
    if constexpr (R == 8) {
        dft8<SIGN>(v);
    } else if constexpr (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

// Radix for the remaining length: 8 when log2 is a multiple of 3, else 4
// (so 16 = 4*4, 32 = 4*8, 128 = 4*4*8 ...), 2 only for a remaining 2.
__host__ __device__ constexpr int pick_radix(int rem) {
    return rem == 2 ? 2 : (ilog2c(rem) % 3 == 0 ? 8 : 4);
}

// Twiddle table tw[t] = exp(SIGN 2 pi i t / L), t < L.
template <int L, int SIGN>
__device__ __forceinline__ void fill_twiddles(float2 *tw, int tid, int nt) {
    for (int t = tid; t < L; t += nt) {
        float s, c;
        sincospif(2.0f * (float)t / (float)L, &s, &c);
        tw[t] = make_float2(c, SIGN * s);
    }
}

template <int L, int R, int NS, int C, int P, int NT, int SIGN>
__device__ __forceinline__ void fft_pass(float2 *buf, const float2 *tw) {
    constexpr int NJ = L / R;
    constexpr int TOTAL = NJ * C;
    constexpr int ITEMS = (TOTAL + NT - 1) / NT;
    const int tid = threadIdx.x;
    float2 v[ITEMS][R];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int item = tid + it * NT;
        if (TOTAL % NT == 0 || item < TOTAL) {
            const int j = item / C, c = item - (item / C) * C;
#pragma unroll
            for (int r = 0; r < R; ++r) v[it][r] = buf[(j + r * NJ) * P + c];
            if constexpr (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], tw[r * k * (L / (NS * R))]);
            }
            dft_r<R, SIGN>(v[it]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int item = tid + it * NT;
        if (TOTAL % NT == 0 || item < TOTAL) {
            const int j = item / C, c = item - (item / C) * C;
            const int k = j % NS;
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(base + r * NS) * P + c] = v[it][r];
        }
    }
    __syncthreads();
}

template <int L, int NS, int C, int P, int NT, int SIGN>
struct FftRun {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tw) {
        if constexpr (NS < L) {
            constexpr int R = pick_radix(L / NS);
            fft_pass<L, R, NS, C, P, NT, SIGN>(buf, tw);
            FftRun<L, NS * R, C, P, NT, SIGN>::run(buf, tw);
        }
    }
};

// Row pitch (in complex elements) of a tile with C columns: one extra element
// when a warp spans several rows, so that the rows a warp touches in one
// access fall on different shared-memory banks.
__host__ __device__ constexpr int fft_pitch(int C) { return C >= 32 ? C : C + 1; }

// Transform all C columns of buf[L][P] (row pitch P >= C) in place.  Every
// thread of the block (NT of them) must call it; the caller synchronises
// before the first call.
template <int L, int C, int NT, int SIGN, int P = fft_pitch(C)>
__device__ __forceinline__ void smem_fft(float2 *buf, const float2 *tw) {
    FftRun<L, 1, C, P, NT, SIGN>::run(buf, tw);
}

}  // namespace mmsar
