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

#include <utility>

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

// ---------------------------------------------------------------- register DFTs
// N-point DFTs held entirely in one thread's registers (N = 2 .. 64), with
// every internal twiddle a compile-time constant.  N > 8 splits as
// N = R1 x N2 (R1 = 4 for N = 16, else 8): R1-point DFTs over the N2
// decimated subsequences, twiddles exp(SIGN 2 pi i n2 k1 / N), then N2-point
// DFTs, X[k1 + R1 k2] = sum_n2 W_N2^(n2 k2) W_N^(n2 k1) sum_n1 x[n2 + N2 n1] W_R1^(n1 k1).

// cos / sin of 2 pi m / n (exact multiples of a turn), evaluated at compile
// time: reduce to [0, pi/4] by the octant symmetries, then Taylor series.
__host__ __device__ constexpr double ct_sin_series(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos_series(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
// (cos, sin)(2 pi m / n) for m in [0, n): eighth-turn octants o = 0..7
__host__ __device__ constexpr double ct_cos_turn(int m, int n) {
    const double pi = 3.141592653589793238462643383279502884;
    const int e = 8 * m / n;                      // octant
    const double r = (double)(8 * m - e * n) / n; // position inside it, [0, 1)
    const double a = (pi / 4.0) * r, b = (pi / 4.0) * (1.0 - r);
    switch (e) {
        case 0: return ct_cos_series(a);
        case 1: return ct_sin_series(b);
        case 2: return -ct_sin_series(a);
        case 3: return -ct_cos_series(b);
        case 4: return -ct_cos_series(a);
        case 5: return -ct_sin_series(b);
        case 6: return ct_sin_series(a);
        default: return ct_cos_series(b);
    }
}
__host__ __device__ constexpr double ct_sin_turn(int m, int n) {
    // sin(theta) = cos(theta - pi/2): shift by a quarter turn
    return ct_cos_turn(((4 * m - n) % (4 * n) + 4 * n) % (4 * n), 4 * n);
}

// a * exp(SIGN 2 pi i M / N), M and N compile-time
template <int N, int M, int SIGN>
__device__ __forceinline__ float2 twiddle_ct(float2 a) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == N) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * m == N) {
        return mul_si<SIGN>(a);
    } else if constexpr (4 * m == 3 * N) {
        return mul_si<-SIGN>(a);
    } else {
        constexpr float c = (float)ct_cos_turn(m, N);
        constexpr float s = (float)(SIGN * ct_sin_turn(m, N));
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>()), ...);
}
// f(std::integral_constant<int, i>) for i = 0 .. N-1, unrolled at compile time
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>());
}

// In-place DFT of v[0..N-1] (natural order in and out).
template <int N, int SIGN>
__device__ __forceinline__ void reg_dft(float2 *v) {
    if constexpr (N <= 8) {
        dft_r<N, SIGN>(v);
    } else {
        constexpr int R1 = N == 16 ? 4 : 8;
        constexpr int N2 = N / R1;
        float2 t[N];
        static_for<N2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            float2 a[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[n2 + N2 * n1];
            dft_r<R1, SIGN>(a);
            static_for<R1>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                t[n2 * R1 + k1] = twiddle_ct<N, n2 * k1, SIGN>(a[k1]);
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 b[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) b[n2] = t[n2 * R1 + k1];
            reg_dft<N2, SIGN>(b);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k1 + R1 * k2] = b[k2];
        }
    }
}

// ---------------------------------------------------------------- column pairs
// Two columns' complex values in split form: re = (re_a, re_b), im =
// (im_a, im_b).  Every packed two-lane instruction then serves both columns,
// and a multiplication by +-i is a swap of the halves folded into the next
// addition.  The DFTs below are those of reg_dft, column by column.
struct cpair {
    float2 re, im;
};
__device__ __forceinline__ cpair padd(cpair a, cpair b) { return {fadd2(a.re, b.re), fadd2(a.im, b.im)}; }
__device__ __forceinline__ cpair psub(cpair a, cpair b) { return {fsub2(a.re, b.re), fsub2(a.im, b.im)}; }
// a + SIGN i b and a - SIGN i b
template <int SIGN>
__device__ __forceinline__ cpair padd_si(cpair a, cpair b) {
    return SIGN > 0 ? cpair{fsub2(a.re, b.im), fadd2(a.im, b.re)} : cpair{fadd2(a.re, b.im), fsub2(a.im, b.re)};
}
template <int SIGN>
__device__ __forceinline__ cpair psub_si(cpair a, cpair b) {
    return SIGN > 0 ? cpair{fadd2(a.re, b.im), fsub2(a.im, b.re)} : cpair{fsub2(a.re, b.im), fadd2(a.im, b.re)};
}
// a (c + i s) with (c, s) broadcast to both columns
__device__ __forceinline__ cpair pmul_cs(cpair a, float c, float s) {
    const float2 cc = make_float2(c, c), ss = make_float2(s, s);
    return {fsub2(fmul2(a.re, cc), fmul2(a.im, ss)), ffma2(a.re, ss, fmul2(a.im, cc))};
}

template <int SIGN>
__device__ __forceinline__ void pdft4(cpair &a0, cpair &a1, cpair &a2, cpair &a3) {
    const cpair t0 = padd(a0, a2), t1 = psub(a0, a2);
    const cpair t2 = padd(a1, a3), d = psub(a1, a3);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    a1 = padd_si<SIGN>(t1, d);   // t1 + SIGN i d
    a3 = psub_si<SIGN>(t1, d);
}

template <int SIGN>
__device__ __forceinline__ void pdft8(cpair *v) {
    cpair e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cpair o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    pdft4<SIGN>(e0, e1, e2, e3);
    pdft4<SIGN>(o0, o1, o2, o3);
    const float2 r = make_float2(0.70710678118654752440f, 0.70710678118654752440f);
    // o1 *= r (1 + SIGN i), o3 *= r (-1 + SIGN i); o2 *= SIGN i folds into the additions
    if (SIGN > 0) {
        o1 = {fmul2(fsub2(o1.re, o1.im), r), fmul2(fadd2(o1.im, o1.re), r)};
        o3 = {fmul2(fadd2(o3.re, o3.im), make_float2(-r.x, -r.y)), fmul2(fsub2(o3.re, o3.im), r)};
    } else {
        o1 = {fmul2(fadd2(o1.re, o1.im), r), fmul2(fsub2(o1.im, o1.re), r)};
        o3 = {fmul2(fsub2(o3.im, o3.re), r), fmul2(fadd2(o3.re, o3.im), make_float2(-r.x, -r.y))};
    }
    v[0] = padd(e0, o0); v[4] = psub(e0, o0);
    v[1] = padd(e1, o1); v[5] = psub(e1, o1);
    v[2] = padd_si<SIGN>(e2, o2); v[6] = psub_si<SIGN>(e2, o2);
    v[3] = padd(e3, o3); v[7] = psub(e3, o3);
}

template <int R, int SIGN>
__device__ __forceinline__ void pdft_r(cpair *v) {
    if constexpr (R == 8) {
        pdft8<SIGN>(v);
    } else if constexpr (R == 4) {
        pdft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else {
        const cpair a = v[0], b = v[1];
        v[0] = padd(a, b);
        v[1] = psub(a, b);
    }
}

// a * exp(SIGN 2 pi i M / N) on a column pair, M and N compile-time
template <int N, int M, int SIGN>
__device__ __forceinline__ cpair ptwiddle_ct(cpair a) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == N) {
        const float2 neg = make_float2(-1.f, -1.f);
        return {fmul2(a.re, neg), fmul2(a.im, neg)};
    } else if constexpr (4 * m == N || 4 * m == 3 * N) {
        // times +-i: (re, im) -> (-+im, +-re)
        constexpr int S = (4 * m == N) ? SIGN : -SIGN;
        const float2 neg = make_float2(-1.f, -1.f);
        return S > 0 ? cpair{fmul2(a.im, neg), a.re} : cpair{a.im, fmul2(a.re, neg)};
    } else {
        constexpr float c = (float)ct_cos_turn(m, N);
        constexpr float s = (float)(SIGN * ct_sin_turn(m, N));
        return pmul_cs(a, c, s);
    }
}

// In-place DFT of v[0..N-1] for both columns of the pairs (natural order in
// and out), the same decomposition as reg_dft.
template <int N, int SIGN>
__device__ __forceinline__ void preg_dft(cpair *v) {
    if constexpr (N <= 8) {
        pdft_r<N, SIGN>(v);
    } else {
        constexpr int R1 = N == 16 ? 4 : 8;
        constexpr int N2 = N / R1;
        cpair t[N];
        static_for<N2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            cpair a[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[n2 + N2 * n1];
            pdft_r<R1, SIGN>(a);
            static_for<R1>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                t[n2 * R1 + k1] = ptwiddle_ct<N, n2 * k1, SIGN>(a[k1]);
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            cpair b[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) b[n2] = t[n2 * R1 + k1];
            preg_dft<N2, SIGN>(b);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k1 + R1 * k2] = b[k2];
        }
    }
}

}  // namespace mmsar
