// Column-batched FFT kernel for the spatial transforms of Eq. 16: the
// forward FT_2D over (x', y') after gridding (with the Gaussian
// deconvolution and the crop to the Mx x My spectrum fused into the store)
// and the inverse transform over (k_x, k_y) (with the crop to the voxel grid
// and the 1/N normalisation fused into the store).
//
// Every transform runs along a strided axis of a tensor whose innermost
// axis is contiguous: a CTA loads L rows x C contiguous columns (coalesced
// rows of C * 8 bytes), transforms the C columns in shared memory (fft.cuh)
// and writes the selected output rows.  No transposes are needed anywhere.
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

constexpr int kFftThreads = 256;

// Columns per tile and row pitch: two tiles (double buffer) of L x P complex
// fit in shared memory; P is even so 16-byte asynchronous copies stay aligned.
__host__ __device__ constexpr int fft_cols(int L) { return L >= 256 ? 8192 / L : 32; }
__host__ __device__ constexpr int fft_tile_pitch(int C) { return C >= 32 ? C : C + 2; }

__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc, bool live, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    const int n = live ? bytes : 0;   // 0 source bytes: the destination is zero-filled
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One tile per CTA: the tile arrives through asynchronous copies (zero-filled
// outside the input window), is transformed in shared memory and the
// selected rows are scaled and stored.  VEC complex values per copy (2 when
// every row start is 16-byte aligned, else 1).
template <int L, int SIGN, int VEC>
__device__ __forceinline__ void column_fft_body(const ColumnFFT &a, int bx, int by) {
    constexpr int C = fft_cols(L);
    constexpr int P = fft_tile_pitch(C);
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem;
    float2 *tw = smem + L * P;
    const int tid = threadIdx.x;
    const int nchunks = (a.ncols + C - 1) / C;
    const int chunk = bx % nchunks;
    const int t2 = bx / nchunks;
    const int t1 = by;
    if (a.tile_win) {
        const int len = a.tile_win[1];
        if (len < a.nt2) {
            int d = (t2 - a.tile_win[0]) % a.nt2;
            if (d < 0) d += a.nt2;
            if (d >= len) return;   // a row that is known to be zero: nothing to do
        }
    }
    int wlo = 0, wlen = a.n_in;
    if (a.in_win) {
        wlo = a.in_win[0];
        wlen = a.in_win[1];
    }
    const int c0 = chunk * C;
    const int cw = min(C, a.ncols - c0);
    const float2 *in = a.in + t1 * a.in_t1 + t2 * a.in_t2 + c0;
    float2 *out = a.out + t1 * a.out_t1 + t2 * a.out_t2 + c0;
    constexpr int PER_ROW = C / VEC;
    for (int e = tid; e < L * PER_ROW; e += kFftThreads) {
        const int f = e / PER_ROW, c = (e - f * PER_ROW) * VEC;
        const int r = (f - a.in_shift) & (L - 1);
        int d = r - wlo;
        if (d < 0) d += a.n_in;
        const bool live = r < a.n_in && c < cw && d < wlen;
        cp_async(tile + f * P + c, live ? in + (long long)r * a.in_row + c : a.in, live, VEC * 8);
    }
    cp_async_commit();
    fill_twiddles<L, SIGN>(tw, tid, kFftThreads);
    cp_async_wait<0>();
    __syncthreads();
    smem_fft<L, C, kFftThreads, SIGN, P>(tile, tw);
    const int half = a.n_out / 2;
    for (int e = tid; e < a.n_out * C; e += kFftThreads) {
        const int o = e / C, c = e - (e / C) * C;
        if (c < cw) {
            const int f = o - half;
            float sc = a.scale;
            if (a.gauss_tau > 0.f) sc *= __expf((float)(f * f) * a.gauss_tau);
            const float2 v = tile[(f & (L - 1)) * P + c];
            out[(long long)o * a.out_row + c] = make_float2(v.x * sc, v.y * sc);
        }
    }
}

// Register kernel (L = 64 .. 1024): the same tile of L rows x C columns as a
// two-step transform, L = N1 x N2.  Step 1: a thread takes input rows
// n2 + N2 n1 (n1 = 0 .. N1-1) of one column straight from global memory into
// registers (all its loads in flight at once), runs the N1-point DFT,
// multiplies by exp(SIGN 2 pi i n2 k1 / L) and writes the N1 results to a
// transpose buffer in shared memory.  Step 2: a thread takes the N2 values
// of one (k1, column), runs the N2-point DFT and stores the kept outputs
// X[k1 + N1 k2] directly.  Shared memory is written once and read once.
__host__ __device__ constexpr int reg_fft_n1(int L) { return L <= 128 ? 8 : (L <= 512 ? 16 : 32); }
__host__ __device__ constexpr int reg_fft_pitch(int L) {
    return reg_fft_n1(L) * fft_cols(L) + (fft_cols(L) < 32 ? 8 : 0);
}

// PAIR: step 1 on pairs of adjacent columns (16-byte loads, the window test
// and the inter-step twiddle shared by the two, the DFT in split form:
// cpair in fft.cuh); needs 16-byte aligned rows and two step-1 columns per
// thread.
template <int L, int SIGN, bool PAIR>
__device__ __forceinline__ void column_fft_reg_body(const ColumnFFT &a, int bx, int by) {
    constexpr int N1 = reg_fft_n1(L), N2 = L / N1;
    constexpr int C = fft_cols(L);
    constexpr int IT1 = N2 * C / kFftThreads;   // step-1 columns per thread (N1 values each)
    constexpr int IT2 = N1 * C / kFftThreads;   // step-2 columns per thread (N2 values each)
    static_assert(IT1 >= 1 && IT2 >= 1 && (N2 * C) % kFftThreads == 0 && (N1 * C) % kFftThreads == 0,
                  "tile does not split evenly over the threads");
    constexpr int YP = reg_fft_pitch(L);   // pitch of one n2 row of the transpose buffer (complex)
    extern __shared__ __align__(16) float2 smem[];
    float2 *y = smem;              // [N2][YP]: y[n2][k1 C + c]
    float2 *tw = smem + N2 * YP;   // [L]: exp(SIGN 2 pi i t / L)
    float *dscale = reinterpret_cast<float *>(tw + L);   // [n_out <= L]: output row scales
    const int tid = threadIdx.x;
    const int nchunks = (a.ncols + C - 1) / C;
    const int chunk = bx % nchunks;
    const int t2 = bx / nchunks;
    const int t1 = by;
    if (a.tile_win) {
        const int len = a.tile_win[1];
        if (len < a.nt2) {
            int d = (t2 - a.tile_win[0]) % a.nt2;
            if (d < 0) d += a.nt2;
            if (d >= len) return;   // a row that is known to be zero: nothing to do
        }
    }
    int wlo = 0, wlen = a.n_in;
    if (a.in_win) {
        wlo = a.in_win[0];
        wlen = a.in_win[1];
    }
    const int c0 = chunk * C;
    const int cw = min(C, a.ncols - c0);
    const float2 *in = a.in + t1 * a.in_t1 + t2 * a.in_t2 + c0;
    float2 *out = a.out + t1 * a.out_t1 + t2 * a.out_t2 + c0;

    // step 1: loads (zero outside the occupied window); all L rows are input
    // rows here (n_in = L), so row r = (f - in_shift) mod L and the window
    // test is (r - wlo) mod L < wlen
    constexpr int IP = PAIR ? IT1 / 2 : 1;   // column pairs per thread
    static_assert(!PAIR || (IT1 % 2 == 0 && C % 2 == 0), "pairs of step-1 columns");
    float2 v[PAIR ? 1 : IT1][N1];
    cpair vp[IP][PAIR ? N1 : 1];
    if constexpr (PAIR) {
#pragma unroll
        for (int it = 0; it < IP; ++it) {
            const int item = tid + it * kFftThreads;
            const int c = 2 * (item % (C / 2)), n2 = item / (C / 2);
            const int r0 = n2 - a.in_shift, d0 = r0 - wlo;
            const bool c0ok = c < cw, c1ok = c + 1 < cw;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int r = (r0 + N2 * n1) & (L - 1);
                const bool live = ((d0 + N2 * n1) & (L - 1)) < wlen;
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                const float2 *src = in + (long long)r * a.in_row + c;
                if (live && c1ok) {
                    t = __ldg(reinterpret_cast<const float4 *>(src));
                } else if (live && c0ok) {
                    const float2 t0 = __ldg(src);
                    t.x = t0.x;
                    t.y = t0.y;
                }
                vp[it][n1] = cpair{make_float2(t.x, t.z), make_float2(t.y, t.w)};
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < IT1; ++it) {
            const int item = tid + it * kFftThreads;
            const int c = item % C, n2 = item / C;
            const int r0 = n2 - a.in_shift, d0 = r0 - wlo;
            const bool cok = c < cw;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int r = (r0 + N2 * n1) & (L - 1);
                const bool live = cok && ((d0 + N2 * n1) & (L - 1)) < wlen;
                v[it][n1] = live ? in[(long long)r * a.in_row + c] : make_float2(0.f, 0.f);
            }
        }
    }
    fill_twiddles<L, SIGN>(tw, tid, kFftThreads);
    // scale of each kept output row: scale * exp(f^2 tau) (Gaussian deconvolution)
    const int half = a.n_out / 2;
    for (int o = tid; o < a.n_out; o += kFftThreads) {
        const int f = o - half;
        dscale[o] = a.gauss_tau > 0.f ? a.scale * expf((float)(f * f) * a.gauss_tau) : a.scale;
    }
    __syncthreads();
    if constexpr (PAIR) {
#pragma unroll
        for (int it = 0; it < IP; ++it) {
            const int item = tid + it * kFftThreads;
            const int c = 2 * (item % (C / 2)), n2 = item / (C / 2);
            preg_dft<N1, SIGN>(vp[it]);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                cpair o = vp[it][k1];
                if (k1 > 0) {
                    const float2 w = tw[(n2 * k1) & (L - 1)];
                    o = pmul_cs(o, w.x, w.y);
                }
                *reinterpret_cast<float4 *>(y + n2 * YP + k1 * C + c) = make_float4(o.re.x, o.im.x, o.re.y, o.im.y);
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < IT1; ++it) {
            const int item = tid + it * kFftThreads;
            const int c = item % C, n2 = item / C;
            reg_dft<N1, SIGN>(v[it]);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1)
                y[n2 * YP + k1 * C + c] = k1 == 0 ? v[it][0] : cmul(v[it][k1], tw[(n2 * k1) & (L - 1)]);
        }
    }
    __syncthreads();

    // step 2: N2-point DFTs and the stores of the kept rows
#pragma unroll
    for (int it = 0; it < IT2; ++it) {
        const int item = tid + it * kFftThreads;
        const int c = item % C, k1 = item / C;
        float2 b[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) b[n2] = y[n2 * YP + k1 * C + c];
        reg_dft<N2, SIGN>(b);
        if (c < cw) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int i = k1 + N1 * k2;                      // FFT output index
                const int o = (i < L / 2 ? i : i - L) + half;    // signed frequency + half
                if (o >= 0 && o < a.n_out) {
                    const float sc = dscale[o];
                    out[(long long)o * a.out_row + c] = fmul2(make_float2(sc, sc), b[k2]);
                }
            }
        }
    }
}

template <int L, int SIGN, int VEC>
__global__ void __launch_bounds__(kFftThreads) column_fft_kernel(const __grid_constant__ ColumnFFT a) {
    column_fft_body<L, SIGN, VEC>(a, blockIdx.x, blockIdx.y);
}
// three CTAs per SM, as the tiles' shared memory allows
template <int L, int SIGN, bool PAIR>
__global__ void __launch_bounds__(kFftThreads, 3)
    column_fft_reg_kernel(const __grid_constant__ ColumnFFT a) {
    column_fft_reg_body<L, SIGN, PAIR>(a, blockIdx.x, blockIdx.y);
}

// Fused launches: the tiles of every scan on a 1-D grid (x fastest as above).
template <int L, int SIGN, int VEC>
__global__ void __launch_bounds__(kFftThreads)
    column_fft_multi(const __grid_constant__ BatchTable<ColumnFFT> t) {
    __shared__ ColumnFFT sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    const int gx = sa.nt2 * ((sa.ncols + fft_cols(L) - 1) / fft_cols(L));
    column_fft_body<L, SIGN, VEC>(sa, bid % gx, bid / gx);
}
template <int L, int SIGN, bool PAIR>
__global__ void __launch_bounds__(kFftThreads, 3)
    column_fft_reg_multi(const __grid_constant__ BatchTable<ColumnFFT> t) {
    __shared__ ColumnFFT sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    const int gx = sa.nt2 * ((sa.ncols + fft_cols(L) - 1) / fft_cols(L));
    column_fft_reg_body<L, SIGN, PAIR>(sa, bid % gx, bid / gx);
}

// Kernel instance of a transform: bit 0-1 the kind (0 / 3 the register
// kernel, 3 with step 1 on column pairs; 1 / 2 the shared-memory kernel with
// 8- / 16-byte copies), bits 2.. L, bit 20 the inverse sign.
static int fft_key(const ColumnFFT &a) {
    const bool reg = a.n_in == a.L && a.L >= 64 && a.L <= 1024;
    // 16-byte copies need every row start (and the column chunk starts) on a
    // 16-byte boundary
    const bool even = (a.ncols % 2 == 0) && (a.in_row % 2 == 0) && (a.in_t1 % 2 == 0) && (a.in_t2 % 2 == 0) &&
                      (reinterpret_cast<uintptr_t>(a.in) % 16 == 0);
    // column pairs in step 1 where every thread takes two step-1 columns
    const bool pair = reg && even && a.L >= 128 && a.L <= 512;
    return (a.sign > 0 ? 1 << 20 : 0) | (a.L << 2) | (reg ? (pair ? 3 : 0) : (even ? 2 : 1));
}

static int fft_blocks(const ColumnFFT &a) {
    if (a.nt1 <= 0 || a.nt2 <= 0 || a.ncols <= 0) return 0;
    const int C = fft_cols(a.L);
    return a.nt1 * a.nt2 * ((a.ncols + C - 1) / C);
}

template <int L, int SIGN, bool PAIR>
static cudaError_t launch_reg(const ColumnFFT *a, const BatchTable<ColumnFFT> *t, int blocks, cudaStream_t s) {
    constexpr int C = fft_cols(L);
    const size_t smem = (size_t)((L / reg_fft_n1(L)) * reg_fft_pitch(L) + L) * sizeof(float2) + L * sizeof(float);
    if (a) {
        cudaError_t e = ensure_smem_attr((const void *)column_fft_reg_kernel<L, SIGN, PAIR>, smem);
        if (e != cudaSuccess) return e;
        const int nchunks = (a->ncols + C - 1) / C;
        dim3 grid((unsigned)(a->nt2 * nchunks), (unsigned)a->nt1);
        column_fft_reg_kernel<L, SIGN, PAIR><<<grid, kFftThreads, smem, s>>>(*a);
    } else {
        cudaError_t e = ensure_smem_attr((const void *)column_fft_reg_multi<L, SIGN, PAIR>, smem);
        if (e != cudaSuccess) return e;
        column_fft_reg_multi<L, SIGN, PAIR><<<blocks, kFftThreads, smem, s>>>(*t);
    }
    return cudaGetLastError();
}

template <int L, int SIGN, int VEC>
static cudaError_t launch_LV(const ColumnFFT *a, const BatchTable<ColumnFFT> *t, int blocks, cudaStream_t s) {
    constexpr int C = fft_cols(L);
    const size_t smem = (size_t)(L * fft_tile_pitch(C) + L) * sizeof(float2);
    if (a) {
        cudaError_t e = ensure_smem_attr((const void *)column_fft_kernel<L, SIGN, VEC>, smem);
        if (e != cudaSuccess) return e;
        const int nchunks = (a->ncols + C - 1) / C;
        dim3 grid((unsigned)(a->nt2 * nchunks), (unsigned)a->nt1);
        column_fft_kernel<L, SIGN, VEC><<<grid, kFftThreads, smem, s>>>(*a);
    } else {
        cudaError_t e = ensure_smem_attr((const void *)column_fft_multi<L, SIGN, VEC>, smem);
        if (e != cudaSuccess) return e;
        column_fft_multi<L, SIGN, VEC><<<blocks, kFftThreads, smem, s>>>(*t);
    }
    return cudaGetLastError();
}

template <int L, int SIGN>
static cudaError_t launch_kind(int kind, const ColumnFFT *a, const BatchTable<ColumnFFT> *t, int blocks,
                               cudaStream_t s) {
    if constexpr (L >= 128 && L <= 512)
        if (kind == 3) return launch_reg<L, SIGN, true>(a, t, blocks, s);
    if constexpr (L >= 64 && L <= 1024)
        if (kind == 0) return launch_reg<L, SIGN, false>(a, t, blocks, s);
    return kind == 2 ? launch_LV<L, SIGN, 2>(a, t, blocks, s) : launch_LV<L, SIGN, 1>(a, t, blocks, s);
}

template <int SIGN>
static cudaError_t dispatch(int L, int kind, const ColumnFFT *a, const BatchTable<ColumnFFT> *t, int blocks,
                            cudaStream_t s) {
    switch (L) {
        case 16: return launch_kind<16, SIGN>(kind, a, t, blocks, s);
        case 32: return launch_kind<32, SIGN>(kind, a, t, blocks, s);
        case 64: return launch_kind<64, SIGN>(kind, a, t, blocks, s);
        case 128: return launch_kind<128, SIGN>(kind, a, t, blocks, s);
        case 256: return launch_kind<256, SIGN>(kind, a, t, blocks, s);
        case 512: return launch_kind<512, SIGN>(kind, a, t, blocks, s);
        case 1024: return launch_kind<1024, SIGN>(kind, a, t, blocks, s);
        case 2048: return launch_kind<2048, SIGN>(kind, a, t, blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_key(int key, const ColumnFFT *a, const BatchTable<ColumnFFT> *t, int blocks,
                              cudaStream_t s) {
    const int L = (key >> 2) & 0x3ffff, kind = key & 3;
    return (key >> 20) ? dispatch<+1>(L, kind, a, t, blocks, s) : dispatch<-1>(L, kind, a, t, blocks, s);
}

cudaError_t launch_column_fft(const ColumnFFT &a, cudaStream_t s) {
    if (fft_blocks(a) == 0) return cudaSuccess;
    return launch_key(fft_key(a), &a, nullptr, 0, s);
}

// ---------------------------------------------------------------- FT_2D
static ColumnFFT fft_x_args(const Plan &p, void *ws) {
    char *w = reinterpret_cast<char *>(ws);
    const float2 *G = reinterpret_cast<const float2 *>(w + p.off_G);
    float2 *A = reinterpret_cast<float2 *>(w + p.off_A);
    // along x': G[kc][v][u][32] -> A[kc][v][m][32], Gaussian deconvolution in x
    ColumnFFT u;
    u.L = p.mrx;
    u.sign = -1;
    u.in = G;
    u.out = A;
    u.n_in = p.mrx;
    u.in_shift = 0;
    u.in_row = kKC;
    u.in_t1 = (long long)p.mry * p.mrx * kKC;
    u.in_t2 = (long long)p.mrx * kKC;
    u.n_out = p.mx;
    u.out_row = kKC;
    u.out_t1 = (long long)p.mry * p.mx * kKC;
    u.out_t2 = (long long)p.mx * kKC;
    u.ncols = kKC;
    u.nt1 = p.n_kc;
    u.nt2 = p.mry;
    u.scale = (float)(std::sqrt(kPi / p.tau_x) / p.mrx);
    u.gauss_tau = (float)p.tau_x;
    const WsHeader *hdr = reinterpret_cast<const WsHeader *>(w);
    u.in_win = &hdr->u_lo;     // cells of a row outside the occupied window are zero
    u.tile_win = &hdr->v_lo;   // rows outside it are zero: skipped, A left unwritten
    return u;
}

static ColumnFFT fft_y_args(const Plan &p, void *ws) {
    char *w = reinterpret_cast<char *>(ws);
    const float2 *A = reinterpret_cast<const float2 *>(w + p.off_A);
    float2 *S = reinterpret_cast<float2 *>(w + p.off_S);
    // along y': A[kc][v][m][32] -> S[m][n][k], Gaussian deconvolution in y
    ColumnFFT v;
    v.L = p.mry;
    v.sign = -1;
    v.in = A;
    v.out = S;
    v.n_in = p.mry;
    v.in_shift = 0;
    v.in_row = (long long)p.mx * kKC;
    v.in_t1 = (long long)p.mry * p.mx * kKC;
    v.in_t2 = kKC;
    v.n_out = p.my;
    v.out_row = p.nkp;
    v.out_t1 = kKC;
    v.out_t2 = (long long)p.my * p.nkp;
    v.ncols = kKC;
    v.nt1 = p.n_kc;
    v.nt2 = p.mx;
    v.scale = (float)(std::sqrt(kPi / p.tau_y) / p.mry);
    v.gauss_tau = (float)p.tau_y;
    v.in_win = &reinterpret_cast<const WsHeader *>(w)->v_lo;   // only the occupied rows of A
    v.tile_win = nullptr;
    return v;
}

// ---------------------------------------------------------------- IFT over (k_x, k_y)
static ColumnFFT ifft_y_args(const Plan &p, void *ws) {
    char *w = reinterpret_cast<char *>(ws);
    const float2 *Z = reinterpret_cast<const float2 *>(w + p.off_Z);
    float2 *B = reinterpret_cast<float2 *>(w + p.off_B);
    const int ny = p.grid.ny, nz = p.grid.nz;
    // along k_y: Z[m][n][q] -> B[m][j][q]
    ColumnFFT a;
    a.L = p.my;
    a.sign = +1;
    a.in = Z;
    a.out = B;
    a.n_in = p.my;
    a.in_shift = p.my / 2;
    a.in_row = nz;
    a.in_t1 = 0;
    a.in_t2 = (long long)p.my * nz;
    a.n_out = ny;
    a.out_row = nz;
    a.out_t1 = 0;
    a.out_t2 = (long long)ny * nz;
    a.ncols = nz;
    a.nt1 = 1;
    a.nt2 = p.mx;
    a.scale = 1.0f;
    a.gauss_tau = 0.f;
    a.in_win = nullptr;
    a.tile_win = nullptr;
    return a;
}

static ColumnFFT ifft_x_args(const Plan &p, void *ws, void *vol) {
    char *w = reinterpret_cast<char *>(ws);
    const float2 *B = reinterpret_cast<const float2 *>(w + p.off_B);
    const int nx = p.grid.nx, ny = p.grid.ny, nz = p.grid.nz;
    // along k_x: B[m][j][q] -> vol[i][j][q], 1 / (T R P Nk)
    ColumnFFT b;
    b.L = p.mx;
    b.sign = +1;
    b.in = B;
    b.out = reinterpret_cast<float2 *>(vol);
    b.n_in = p.mx;
    b.in_shift = p.mx / 2;
    b.in_row = (long long)ny * nz;
    b.in_t1 = 0;
    b.in_t2 = nz;
    b.n_out = nx;
    b.out_row = (long long)ny * nz;
    b.out_t1 = 0;
    b.out_t2 = nz;
    b.ncols = nz;
    b.nt1 = 1;
    b.nt2 = ny;
    b.scale = (float)(1.0 / ((double)p.L * p.shape.n_k));
    b.gauss_tau = 0.f;
    b.in_win = nullptr;
    b.tile_win = nullptr;
    return b;
}

cudaError_t launch_fft_x(const Plan &p, void *ws, cudaStream_t s) { return launch_column_fft(fft_x_args(p, ws), s); }
cudaError_t launch_fft_y(const Plan &p, void *ws, cudaStream_t s) { return launch_column_fft(fft_y_args(p, ws), s); }
cudaError_t launch_ifft_y(const Plan &p, void *ws, cudaStream_t s) { return launch_column_fft(ifft_y_args(p, ws), s); }
cudaError_t launch_ifft_x(const Plan &p, void *ws, void *vol, cudaStream_t s) {
    return launch_column_fft(ifft_x_args(p, ws, vol), s);
}

// stage 0: along x', 1: along y', 2: inverse along k_y, 3: inverse along k_x
cudaError_t launch_fft_multi(const mmsar_request *r, int n, int stage, cudaStream_t s) {
    std::vector<ColumnFFT> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n);
    for (int i = 0; i < n; ++i) {
        const Plan &p = r[i].plan->p;
        void *ws = r[i].workspace;
        args[i] = stage == 0 ? fft_x_args(p, ws)
                  : stage == 1 ? fft_y_args(p, ws)
                  : stage == 2 ? ifft_y_args(p, ws)
                               : ifft_x_args(p, ws, r[i].vol);
        blocks[i] = fft_blocks(args[i]);
        keys[i] = fft_key(args[i]);
    }
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int key, const BatchTable<ColumnFFT> &t, int total) {
                             return launch_key(key, nullptr, &t, total, s);
                         });
}

}  // namespace mmsar
