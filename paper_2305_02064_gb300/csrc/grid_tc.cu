// Gaussian gridding (the spreading step of the fast Gaussian gridding NUFFT
// that Sec. III uses for FT_2D of Eq. 16) on the fifth-generation tensor
// cores, at FP32 accuracy.
//
// For an 8 x 8-cell tile of the 2Mx x 2My periodic aperture grid and one
// group of 64 frequencies, the gridded values are a product
//     G[cell][f] = sum_l w_l(cell) s_hat_l(f),   w_l(u, v) = wx_l(u) wy_l(v),
// over the K samples l whose w x w support meets the tile.  Written with the
// frequencies (re, im interleaved: 128 real columns) as rows,
//     D[128][64 cells] = S^T[128][K] . W^T[K][64 cells],
// it is one tcgen05.mma chain per tile: M = 128, N = 64, K = 16 per
// instruction, FP32 accumulator in tensor memory (64 columns).
//
// FP32 accuracy from FP16 operands: the compensation stage stores every
// sample's row normalised by a power of two 2^a (its largest magnitude in
// [2^13, 2^14); one exponent per sample, all frequencies) as a pair of FP16
// planes, hi = fp16(s 2^a) and lo = fp16(s 2^a - hi); the weights are split
// the same way after the factor 2^(a_ref - a) that undoes the normalisation
// (a_ref = the smallest a of the scan, so the factor is <= 1) is folded into
// them.  Three products per step, hi.hi + hi.lo + lo.hi, are exact in FP32
// (11 x 11-bit significands) and accumulate in FP32: relative error about
// 2^-22 per term, against the largest term of the scan, i.e. what FP32
// arithmetic gives.  The result is multiplied by 2^-a_ref (exact) on the way
// out.
//
// Persistent CTAs take (tile, batch of up to four 64-frequency groups) work
// items in turn; per item:
//  1. list: the samples of the bins that can reach the tile are read in bin
//     order (records written by the in-bin sort: sample index, first cell,
//     cell fractions), the ones whose support meets the tile are kept in
//     that order (deterministic), with their Gaussian weights on the tile's
//     8 columns and 8 rows (the factor 2^(a_ref - a) folded into the rows);
//  2. chunks of CH listed samples: the samples' hi / lo rows of every group
//     of the batch are gathered with cp.async into the MN-major core-matrix
//     layout of the A operands (P chunks ahead), the threads write the split
//     weights once for all groups (B operand), and one thread issues the
//     chunk's MMAs (three per group and K step, one accumulator of 64
//     tensor-memory columns per group); a tcgen05.commit on the stage's
//     mbarrier tells the producers when the stage may be reused;
//  3. the accumulators are read back with tcgen05.ld and stored to G.
// Tensor memory (64 columns per group of the batch) is allocated and the
// stage mbarriers are initialised once per CTA, and released when it has no
// item left.  Every wait on an mbarrier is bounded (about half a second); on
// expiry the CTA records MMSAR_ERR_DEVICE_TIMEOUT in the error word, waits
// for its own copies, frees its tensor memory and stops, and the other CTAs
// stop at their next item.
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.cuh"

namespace mmsar {

struct GridTcArgs {
    const uint4 *shs;          // [n_g][Lmax][2][16] 16-byte pieces: hi, lo planes of 128 halves
    const signed char *sexp;   // [Lmax] normalisation exponents a
    const int *aref;           // [1] max over samples of (127 - a)
    const int4 *trec;          // [Lmax] bin order: (sample, u0 | v0 << 16, fx bits, fy bits)
    const int *offsets;        // [n_bins + 1]
    float2 *G;                 // [n_kc][mry][mrx][32]
    WsHeader *hdr;             // occupied window, error word
    long long Lmax;
    int mrx, mry, nbx, nby, w, n_kc, n_g;
    float kappa;
    int wait_test;             // 1: one MMA thread waits on a barrier nothing completes (timeout test)
};

constexpr int kTcMaxRanges = 16;

// Pipeline configuration of the tensor-core gridding: CH listed samples per
// MMA chunk (16 or 32: one or two K steps), NST shared-memory stages, the
// rows of chunk q + P gathered while chunk q is prepared, CAP listed samples
// per pass (a tile with more runs several passes into the same
// accumulators), GB frequency groups per work item, T threads, MINB CTAs per
// SM.  Per stage: A (S^T) hi, lo of each group = 16 M-blocks x CH samples x
// 16 B; B (W^T) hi, lo = 8 cell rows x CH samples x 16 B, shared by the
// groups.
template <int CH_, int NST_, int P_, int CAP_, int GB_, int T_, int MINB_, bool REG_ = false>
struct TcCfg {
    static constexpr int CH = CH_, NST = NST_, P = P_, CAP = CAP_, GB = GB_, T = T_, MINB = MINB_;
    // REG: the rows of chunk q + 1 are loaded into registers while chunk q is
    // prepared and stored to its stage at the start of the next iteration
    // (P is then 1: one chunk ahead, held in registers, not in a stage)
    static constexpr bool REG = REG_;
    static constexpr int PIECES = GB * CH * 32 / T;   // 16-byte pieces per thread and chunk
    static constexpr int W = T / 32;   // warps
    static_assert(CH == 16 || CH == 32, "one or two K steps per chunk");
    static_assert(P >= 1 && P + 1 <= NST && NST <= 8, "stages");
    static_assert(GB == 1 || GB == 2 || GB == 4, "groups per item");
    static_assert(T == 128 || T == 256, "threads");
    static_assert(CAP >= T, "one round of candidates (one per thread) must fit the list after a flush");
    static_assert((GB * CH) % W == 0, "gather instructions split evenly over the warps");
    static_assert(T >= 2 * kTcMaxRanges / 2 && W <= 8, "range slots and warp counts");
    static constexpr int APlane = 16 * CH * 16;
    static constexpr int AGroup = 2 * APlane;
    static constexpr int BPlane = 8 * CH * 16;
    static constexpr int StageBytes = GB * AGroup + 2 * BPlane;
    static constexpr int ListBytes = CAP * 4 + 16 * CAP * 4;   // indices, weights [16][cap]
    static constexpr size_t Smem = (size_t)NST * StageBytes + ListBytes + 1024;   // + alignment slack
    static constexpr int TmemCols = 64 * GB;
};
// the variants the plan selects (mmsar_tiles.grid_tensor_cores = 1 .. 4)
using TcCfg1 = TcCfg<16, 2, 1, 256, 4, 256, 2, true>;
using TcCfg2 = TcCfg<16, 2, 1, 256, 4, 256, 2>;
using TcCfg3 = TcCfg<16, 4, 2, 256, 2, 256, 2>;
using TcCfg4 = TcCfg<16, 2, 1, 256, 2, 256, 2, true>;
constexpr int kTcMaxThreads = 256;
constexpr long long kTcWaitCycles = 1000000000ll;   // ~0.5 s at 2 GHz

// instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both
// MN-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: core matrices of 8 K-rows x
// 16 bytes; LBO = byte distance of K-adjacent core matrices, SBO = of
// MN-adjacent ones (the MN-major canonical layout)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// the same with the 128-byte swizzle (atoms of 8 K-rows x 128 bytes, 1024-byte
// aligned): LBO = byte distance of MN-adjacent atoms, SBO = of K-adjacent
// 8-row groups
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return tc_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// the same without a compiler memory barrier: the copy's smem destination is
// read only after cp.async.wait_group (which has one) and its global source is
// not written by the kernel, so loads and address arithmetic of later copies
// may be scheduled ahead of it
__device__ __forceinline__ void cp_async16_free(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ bool tile_meets_tc(int t0, int span, int lo, int len, int m) {
    if (len >= m) return true;
    if (len <= 0) return false;
    int d = (t0 - lo) % m;
    if (d < 0) d += m;
    int e = (lo - t0) % m;
    if (e < 0) e += m;
    return d < len || e < span;
}

// hi / lo FP16 split of eight FP32 values, as two 16-byte pieces
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        const float2 af = __half22float2(a);
        const __half2 b = __floats2half2_rn(v[2 * i] - af.x, v[2 * i + 1] - af.y);
        h[i] = *reinterpret_cast<const uint32_t *>(&a);
        l[i] = *reinterpret_cast<const uint32_t *>(&b);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Per CTA state that lives across its tiles: tensor memory, the stage
// mbarriers and their bookkeeping (a commit per MMA chunk on the chunk's
// stage; `pend` bit s: a commit on stage s not yet waited for, `parity` bit
// s: the parity of the phase that commit completes).
struct TcCta {
    uint32_t tmem;
    uint32_t mbar0;      // shared address of the first stage's mbarrier (8 bytes apart)
    uint32_t pend, parity;
    int stage;           // stage of the next chunk
    bool failed;
};

// Wait for the pending commit of stage s, if any (every thread of the CTA).
__device__ __forceinline__ bool tc_stage_drain(TcCta &c, int s) {
    if (!((c.pend >> s) & 1u)) return true;
    const bool ok = mbar_wait_bounded(c.mbar0 + 8u * s, (c.parity >> s) & 1u);
    c.parity ^= 1u << s;
    c.pend &= ~(1u << s);
    return ok;
}

// cp.async.wait_group with a run-time count (the instruction takes an immediate)
__device__ __forceinline__ void cp_async_wait_n(int n) {
    switch (n) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        default: cp_async_wait<4>(); break;
    }
}

// One (tile, group batch) work item: list, MMA chunks, accumulators to G.
// Groups g0 .. g0 + ng - 1 (ng <= GB).
template <class C>
__device__ __forceinline__ void grid_tc_item(const GridTcArgs &a, int g0, int ng, int tile, unsigned char *smem,
                                             TcCta &cta) {
    constexpr int CH = C::CH, NST = C::NST, P = C::P, CAP = C::CAP, GB = C::GB, T = C::T, NW = C::W;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = a.mrx >> 3;
    const int U = (tile % tiles_x) * 8, V = (tile / tiles_x) * 8;
    unsigned char *stages = smem;
    int *lidx = reinterpret_cast<int *>(smem + NST * C::StageBytes);
    float *lw = reinterpret_cast<float *>(lidx + CAP);   // [16][cap]: 8 column weights, 8 row weights
    __shared__ int r_beg[kTcMaxRanges], r_pre[kTcMaxRanges + 1];
    __shared__ int slot_beg[kTcMaxRanges], slot_len[kTcMaxRanges];
    __shared__ int n_ranges_s, wcount[kTcMaxThreads / 32];

    // the candidate bins: first cells u0 in [U - (w - 1), U + 7], v0 likewise;
    // each bin row in reach gives one or two runs of consecutive bins (two
    // where the run wraps around the periodic grid), one thread per run
    const int bu_lo = (U - (a.w - 1)) >> 2, bu_hi = (U + 7) >> 2;   // arithmetic shift: floor
    const int bv_lo = (V - (a.w - 1)) >> 2, bv_hi = (V + 7) >> 2;
    if (tid < kTcMaxRanges) {
        const int rr = tid >> 1, part = tid & 1;
        int beg = 0, len = 0;
        if (bv_lo + rr <= bv_hi) {
            const int row = (((bv_lo + rr) % a.nby) + a.nby) % a.nby;
            const int s0 = ((bu_lo % a.nbx) + a.nbx) % a.nbx;
            const int span = bu_hi - bu_lo + 1;
            const int run0 = min(span, a.nbx - s0);               // bins s0 .. s0 + run0 - 1
            const int first = part == 0 ? s0 : 0, run = part == 0 ? run0 : span - run0;   // then 0 .. rest
            if (run > 0) {
                beg = a.offsets[row * a.nbx + first];
                len = a.offsets[row * a.nbx + first + run] - beg;
            }
        }
        slot_beg[tid] = beg;
        slot_len[tid] = len;
    }
    __syncthreads();
    if (tid == 0) {
        int n = 0, tot = 0;
        for (int k = 0; k < kTcMaxRanges; ++k)
            if (slot_len[k] > 0) {
                r_beg[n] = slot_beg[k];
                r_pre[n] = tot;
                tot += slot_len[k];
                ++n;
            }
        r_pre[n] = tot;
        n_ranges_s = n;
    }
    __syncthreads();
    const int n_ranges = n_ranges_s, total = r_pre[n_ranges];
    const int a_ref = 127 - a.aref[0];
    bool first = true;          // the tile's first MMA overwrites the accumulators
    int issued = 0;             // MMA chunks of this tile

    // gather the S rows of listed samples [base, base + CH) of every group of
    // the batch into stage s (entries past n take sample 0 with zero
    // weights): per group CH x 32 pieces of 16 bytes in CH warp-instructions;
    // instruction i covers 16 samples (half h for CH = 32) and one pair of
    // pieces (plane, M-blocks 2b, 2b + 1); lane = 2 x sample + piece: 32
    // contiguous bytes per lane pair, the 16-byte destinations of one M-block
    // contiguous per sample
    auto gather = [&](int s, int base, int n) {
        const uint32_t st = smem_addr(stages + s * C::StageBytes);
        constexpr int PER = CH;   // warp-instructions per group
#pragma unroll
        for (int r = 0; r < GB * PER / NW; ++r) {
            const int i = warp + NW * r;
            const int gl = i / PER, ii = i - gl * PER;
            if (gl >= ng) continue;
            const int h = CH == 32 ? (ii & 1) : 0, pair = CH == 32 ? (ii >> 1) : ii;
            const int j = 16 * h + (lane >> 1);   // sample slot in the chunk
            const int plane = pair >> 3, mi = 2 * (pair & 7) + (lane & 1);
            const int e = base + j;
            const int l = e < n ? lidx[e] : 0;
            const uint4 *src = a.shs + ((long long)(g0 + gl) * a.Lmax + l) * 32 + plane * 16 + mi;
            cp_async16(st + gl * C::AGroup + plane * C::APlane + mi * (CH * 16) + j * 16, src);
        }
    };
    // register-staged form of the same gather: this thread's pieces of
    // listed samples [base, base + CH) into stg (coalesced 16-byte loads),
    // then from stg into stage s
    auto load_rows = [&](uint4 *stg, int base, int n) {
        constexpr int PER = CH;
#pragma unroll
        for (int r = 0; r < C::PIECES; ++r) {
            const int i = warp + NW * r;
            const int gl = i / PER, ii = i - gl * PER;
            const int h = CH == 32 ? (ii & 1) : 0, pair = CH == 32 ? (ii >> 1) : ii;
            const int j = 16 * h + (lane >> 1);
            const int plane = pair >> 3, mi = 2 * (pair & 7) + (lane & 1);
            const int e = base + j;
            const int l = e < n ? lidx[e] : 0;
            stg[r] = gl < ng ? __ldg(a.shs + ((long long)(g0 + gl) * a.Lmax + l) * 32 + plane * 16 + mi)
                             : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    auto store_rows = [&](const uint4 *stg, int s) {
        unsigned char *st = stages + s * C::StageBytes;
        constexpr int PER = CH;
#pragma unroll
        for (int r = 0; r < C::PIECES; ++r) {
            const int i = warp + NW * r;
            const int gl = i / PER, ii = i - gl * PER;
            if (gl >= ng) continue;
            const int h = CH == 32 ? (ii & 1) : 0, pair = CH == 32 ? (ii >> 1) : ii;
            const int j = 16 * h + (lane >> 1);
            const int plane = pair >> 3, mi = 2 * (pair & 7) + (lane & 1);
            *reinterpret_cast<uint4 *>(st + gl * C::AGroup + plane * C::APlane + mi * (CH * 16) + j * 16) = stg[r];
        }
    };
    // split weights of listed samples [base, base + CH) into stage s (shared
    // by the groups): CH x 8 (sample, cell row) items of 8 cells, each done
    // by HV threads (8 / HV cells each)
    auto weights = [&](int s, int base, int n) {
        unsigned char *bw = stages + s * C::StageBytes + GB * C::AGroup;
        constexpr int ITEMS = CH * 8, HV = T >= 2 * ITEMS ? 2 : 1, NC = 8 / HV;
#pragma unroll
        for (int u = tid; u < ITEMS * HV; u += T) {
            const int item = u % ITEMS, half = u / ITEMS;
            const int j = item % CH, r = item / CH;   // sample slot, cell row
            const int e = base + j;
            float v[8];
            const float wy = e < n ? lw[(8 + r) * CAP + e] : 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = (e < n && i < NC) ? lw[(half * NC + i) * CAP + e] * wy : 0.f;
            uint4 hi, lo;
            split8(v, hi, lo);
            unsigned char *d = bw + r * (CH * 16) + j * 16 + half * (2 * NC);
            if constexpr (HV == 1) {
                *reinterpret_cast<uint4 *>(d) = hi;
                *reinterpret_cast<uint4 *>(d + C::BPlane) = lo;
            } else {
                *reinterpret_cast<uint2 *>(d) = make_uint2(hi.x, hi.y);
                *reinterpret_cast<uint2 *>(d + C::BPlane) = make_uint2(lo.x, lo.y);
            }
        }
    };
    auto issue = [&](int s, bool overwrite) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_addr(stages + s * C::StageBytes);
        const uint32_t bhi = st + GB * C::AGroup, blo = bhi + C::BPlane;
        for (int gl = 0; gl < ng; ++gl) {
            const uint32_t ahi = st + gl * C::AGroup, alo = ahi + C::APlane;
#pragma unroll
            for (int ks = 0; ks < CH / 16; ++ks) {
                const uint32_t o = ks * 256;   // two K-adjacent core matrices of 128 bytes per step
                const uint64_t dah = tc_desc(ahi + o, 128, CH * 16), dal = tc_desc(alo + o, 128, CH * 16);
                const uint64_t dbh = tc_desc(bhi + o, 128, CH * 16), dbl = tc_desc(blo + o, 128, CH * 16);
                const uint32_t d = cta.tmem + 64u * gl;
                tc_mma(d, dah, dbh, (overwrite && ks == 0) ? 0u : 1u);
                tc_mma(d, dah, dbl, 1u);
                tc_mma(d, dal, dbh, 1u);
            }
        }
        tc_commit(cta.mbar0 + 8u * s);
    };
    // the MMA chunks of listed samples [0, n): the rows of chunk q + P are
    // gathered while chunk q's weights are written; a stage is reused once
    // its previous commit has been waited for (a thread whose wait expired
    // stops filling stages; the CTA agrees on giving up at the barrier
    // before the next MMA issue)
    auto run_list = [&](int n) {
        const int nch = (n + CH - 1) / CH;
        if (nch == 0 || cta.failed) return;
        const int s0 = cta.stage;
        bool bad = false;
        if constexpr (C::REG) {
            // chunk q: its rows (loaded last iteration) into stage q % NST once
            // the MMAs of chunk q - NST are done, the next chunk's rows into
            // registers, the weights, then the MMAs
            uint4 stg[C::PIECES];
            load_rows(stg, 0, n);
            for (int q = 0; q < nch; ++q) {
                const int s = (s0 + q) % NST;
                if (!tc_stage_drain(cta, s)) bad = true;
                if (!bad) store_rows(stg, s);
                if (q + 1 < nch) load_rows(stg, (q + 1) * CH, n);
                weights(s, q * CH, n);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (__syncthreads_or(bad)) { cta.failed = true; break; }
                if (tid == 0) issue(s, first);
                cta.pend |= 1u << s;
                first = false;
                ++issued;
            }
            cta.stage = (s0 + nch) % NST;
            return;
        }
        const int npre = nch < P ? nch : P;
        for (int q = 0; q < npre; ++q) {
            const int s = (s0 + q) % NST;
            if (!tc_stage_drain(cta, s)) bad = true;
            if (!bad) gather(s, q * CH, n);
            cp_async_commit();
        }
        for (int q = 0; q < nch; ++q) {
            const int s = (s0 + q) % NST;
            if (q + P < nch) {
                const int sp = (s0 + q + P) % NST;
                if (!tc_stage_drain(cta, sp)) bad = true;
                if (!bad) gather(sp, (q + P) * CH, n);
                cp_async_commit();
            }
            weights(s, q * CH, n);
            const int later = (nch - 1 - q) < P ? (nch - 1 - q) : P;   // groups committed after chunk q's
            cp_async_wait_n(later);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (__syncthreads_or(bad)) { cta.failed = true; break; }
            if (tid == 0) issue(s, first);
            cta.pend |= 1u << s;
            first = false;
            ++issued;
        }
        cp_async_wait<0>();
        cta.stage = (s0 + nch) % NST;
    };

    // 1 + 2: list the reaching samples T candidates at a time (the next
    // round's records loaded a round ahead), run chunks whenever the list is
    // full
    auto record = [&](int c) {
        if (c >= total) return make_int4(0, 0, 0, 0);
        int k = 0;
        while (k + 1 < n_ranges && r_pre[k + 1] <= c) ++k;
        return __ldg(a.trec + r_beg[k] + (c - r_pre[k]));
    };
    int n_list = 0;
    int4 rec_next = record(tid);
    for (int base = 0; base < total && !cta.failed; base += T) {
        const int c = base + tid;
        const int4 rec = rec_next;
        rec_next = record(c + T);
        bool keep = false;
        int l = 0, du = 0, dv = 0;
        float fx = 0.f, fy = 0.f;
        if (c < total) {
            l = rec.x;
            du = (rec.y & 0xffff) - U;
            dv = (rec.y >> 16) - V;
            if (du < -(a.mrx >> 1)) du += a.mrx;
            if (du >= (a.mrx >> 1)) du -= a.mrx;
            if (dv < -(a.mry >> 1)) dv += a.mry;
            if (dv >= (a.mry >> 1)) dv -= a.mry;
            fx = __int_as_float(rec.z);
            fy = __int_as_float(rec.w);
            keep = du >= -(a.w - 1) && du <= 7 && dv >= -(a.w - 1) && dv <= 7;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        int before = 0, round = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            before += i < warp ? wcount[i] : 0;
            round += wcount[i];
        }
        __syncthreads();   // wcount read by all before the next round writes it
        if (n_list + round > CAP) {
            run_list(n_list);
            n_list = 0;
            __syncthreads();   // the list may be overwritten
        }
        if (keep) {
            const int e = n_list + before + __popc(m & ((1u << lane) - 1u));
            lidx[e] = l;
            // Gaussian weights exp(-kappa (f - tap)^2) on the tile's columns
            // and rows (tap = cell - first cell, zero outside 0 .. w - 1)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int tap = i - du;
                const float dlt = fx - (float)tap;
                lw[i * CAP + e] = (tap >= 0 && tap < a.w) ? expf(-a.kappa * dlt * dlt) : 0.f;
            }
            const float scale = ldexpf(1.0f, a_ref - (int)a.sexp[l]);   // 2^(a_ref - a) <= 1, exact
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int tap = i - dv;
                const float dlt = fy - (float)tap;
                lw[(8 + i) * CAP + e] = (tap >= 0 && tap < a.w) ? expf(-a.kappa * dlt * dlt) * scale : 0.f;
            }
        }
        n_list += round;
        __syncthreads();
    }
    run_list(n_list);

    // 3: every commit of the tile waited for, then the accumulators to G
    // (x 2^-a_ref); a tile that listed nothing is zero
    bool ok = !cta.failed;
    for (int s = 0; s < NST; ++s)
        if (!tc_stage_drain(cta, s)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        cta.failed = true;
        if (tid == 0) atomicOr(&a.hdr->error, kErrTimeout);
        return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // a warp reads tensor-memory lanes 32 (warp % 4) .. + 31: lane (row)
    // m = 32 (warp % 4) + lane is frequency 64 g + m / 2, component m % 2;
    // with eight warps, warps 0-3 and 4-7 take alternate groups
    const int mrow = 32 * (warp & 3) + lane;
    const float unscale = ldexpf(1.0f, -a_ref);
    for (int gl = warp >> 2; gl < ng; gl += NW / 4) {
        const int f = 64 * (g0 + gl) + (mrow >> 1);
        const int kc = f >> 5;
        const bool live = kc < a.n_kc;
        float *gp = live ? reinterpret_cast<float *>(a.G + (long long)kc * a.mry * a.mrx * kKC) + 2 * (f & 31) +
                               (mrow & 1)
                         : nullptr;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            uint32_t r[16];
            if (issued > 0) {
                // the load writes its registers asynchronously: the wait is in
                // the same statement, so the compiler sees them defined only
                // after it (and cannot reuse them in between)
                const uint32_t taddr = cta.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * gl + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n\ttcgen05.wait::ld.sync.aligned;"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) r[i] = 0u;
            }
            if (live) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = c0 + i, row = n >> 3, col = n & 7;   // cell (U + col, V + row)
                    gp[((long long)(V + row) * a.mrx + (U + col)) * (2 * kKC)] = __uint_as_float(r[i]) * unscale;
                }
            }
        }
    }
    // the accumulators are read by every warp before the next tile overwrites them
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

// Does a tile lie inside the occupied window of the gridding grid?  Tiles
// outside it stay unwritten (the FFT along x' reads only the window and
// takes the rest as zero).
__device__ __forceinline__ bool tc_item_live(const GridTcArgs &a, int tile) {
    const int tiles_x = a.mrx >> 3;
    return tile_meets_tc((tile % tiles_x) * 8, 8, a.hdr->u_lo, a.hdr->u_len, a.mrx) &&
           tile_meets_tc((tile / tiles_x) * 8, 8, a.hdr->v_lo, a.hdr->v_len, a.mry);
}

// CTA set-up and tear-down around a persistent loop: tensor memory (COLS
// columns, a power of two >= 32) allocated and the stage mbarriers
// initialised once, both released when the CTA is done (mbarriers
// invalidated, memory freed).
template <int NST, int COLS>
__device__ __forceinline__ void tc_cta_begin(TcCta &cta, unsigned long long *mbar, uint32_t *tmem_slot) {
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[s])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    cta.tmem = *tmem_slot;
    cta.mbar0 = smem_addr(&mbar[0]);
    cta.pend = 0u;
    cta.parity = 0u;
    cta.stage = 0;
    cta.failed = false;
}

template <int NST, int COLS>
__device__ __forceinline__ void tc_cta_end(TcCta &cta, unsigned long long *mbar) {
    const int tid = threadIdx.x, warp = tid >> 5;
    // every commit is waited for after each tile; a CTA that gave up waits
    // for its own copies (done in run_list) and releases what it holds
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !cta.failed)
        for (int s = 0; s < NST; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&mbar[s])) : "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cta.tmem), "r"(COLS));
}

// Persistent over the work items of one scan (batch-major: item = gb x
// tiles + tile, groups gb GB .. gb GB + GB - 1): CTA b takes items b,
// b + grid, ...
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) grid_tc_kernel(const __grid_constant__ GridTcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long mbar[C::NST];
    __shared__ uint32_t tmem_slot;
    TcCta cta;
    tc_cta_begin<C::NST, C::TmemCols>(cta, mbar, &tmem_slot);
    const int n_tiles = (a.mrx >> 3) * (a.mry >> 3);
    const int n_gb = (a.n_g + C::GB - 1) / C::GB;
    const int items = n_tiles * n_gb;
    for (int it = blockIdx.x; it < items && !cta.failed; it += gridDim.x) {
        // after a wait of another CTA has expired the image is void: stop
        // (one decision for the whole CTA)
        if (__syncthreads_or(*reinterpret_cast<volatile const int *>(&a.hdr->error) & kErrTimeout)) break;
        const int gb = it / n_tiles, tile = it - gb * n_tiles;
        if (!tc_item_live(a, tile)) continue;
        const int g0 = gb * C::GB;
        grid_tc_item<C>(a, g0, min(C::GB, a.n_g - g0), tile, smem, cta);
    }
    tc_cta_end<C::NST, C::TmemCols>(cta, mbar);
}

// Fused batch: the work items of all scans of the table in one index space
// (scan i owns items start[i] .. start[i + 1] - 1), persistent CTAs.
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) grid_tc_multi(const __grid_constant__ BatchTable<GridTcArgs> t) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long mbar[C::NST];
    __shared__ uint32_t tmem_slot;
    __shared__ GridTcArgs sa;
    __shared__ int cur_scan;
    TcCta cta;
    tc_cta_begin<C::NST, C::TmemCols>(cta, mbar, &tmem_slot);
    if (threadIdx.x == 0) cur_scan = -1;
    __syncthreads();
    const int items = t.start[t.n];
    for (int it = blockIdx.x; it < items && !cta.failed; it += gridDim.x) {
        int lo = 0, hi = t.n;   // the scan of this item
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t.start[mid] <= it) lo = mid; else hi = mid;
        }
        if (lo != cur_scan) {   // (uniform) load the scan's arguments
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(&t.a[lo]);
            int *d = reinterpret_cast<int *>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(GridTcArgs) / 4); i += blockDim.x) d[i] = src[i];
            if (threadIdx.x == 0) cur_scan = lo;
            __syncthreads();
        }
        if (__syncthreads_or(*reinterpret_cast<volatile const int *>(&sa.hdr->error) & kErrTimeout)) continue;
        const int local = it - t.start[lo];
        const int n_tiles = (sa.mrx >> 3) * (sa.mry >> 3);
        const int gb = local / n_tiles, tile = local - gb * n_tiles;
        if (!tc_item_live(sa, tile)) continue;
        const int g0 = gb * C::GB;
        grid_tc_item<C>(sa, g0, min(C::GB, sa.n_g - g0), tile, smem, cta);
    }
    tc_cta_end<C::NST, C::TmemCols>(cta, mbar);
}

// ---------------------------------------------------------------------------
// Warp-specialised form (grid_tensor_cores = 5).  One persistent CTA per SM
// runs four roles concurrently, connected by mbarriers, so that listing the
// next tile, gathering rows, the MMAs and the read-back of the previous
// tile overlap instead of taking turns:
//   warps 0-1    MMA issue (one thread each, alternate frequency groups):
//                wait for a filled stage, issue the chunk's MMAs into the
//                tile's accumulator, commit the stage back to the producers
//                and, after a tile's last chunk, the accumulator to the
//                epilogue;
//   warps 2-5    list: the tile's candidate records in bin order, the kept
//                samples and their Gaussian weights, into one of two list
//                buffers (a tile with more than CAP samples fills several
//                segments, accumulated into the same accumulator);
//   warps 6-9    epilogue: accumulator (tcgen05.ld) x 2^-a_ref to G, then the
//                accumulator is released to the MMA warps;
//   warps 10-13  producers: per chunk of CH listed samples, the split weights
//                and the rows of every group of the item by cp.async (whole
//                128-byte lines) into a free stage; each thread arrives on
//                the stage's barrier once after its weight stores and once
//                more, by the copy unit, when its copies have landed
//                (cp.async.mbarrier.arrive.noinc), so a chunk is handed over
//                as soon as its data is there; the MMA threads make the
//                landed copies visible to the tensor cores with a proxy fence
//                after their wait.
// Two accumulators of GB x 64 tensor-memory columns alternate between tiles.
// The A operands (sample rows) use the 128-byte-swizzled MN-major layout,
// the B operands (weights) the unswizzled one.  The chunking (CH consecutive
// list entries, zero weights past the end of a segment) and the MMA order
// are those of the forms above; the list segments differ (a round of
// candidates is 128 records here), so the sums agree with them to rounding,
// and the form is deterministic.
// Every wait is bounded and also ends when another role has given up (a
// shared abort flag); decisions the list warps take together go through a
// barrier reduction, so no thread is left at a named barrier.
constexpr int kWsMmaWarps = 2, kWsListWarps = 4, kWsEpiWarps = 4, kWsProdWarps = 4;
constexpr int kWsWarps = kWsMmaWarps + kWsListWarps + kWsEpiWarps + kWsProdWarps;
constexpr int kWsT = 32 * kWsWarps;                       // 448 threads
constexpr int kWsListT = 32 * kWsListWarps, kWsProdT = 32 * kWsProdWarps;
constexpr int kWsListBar = 1;                             // named barrier of the list warps

template <int NST_, int CAP_, int GB_>
struct WsCfg {
    static constexpr int CH = 16, NST = NST_, CAP = CAP_, GB = GB_;
    static_assert(NST >= 2 && NST <= 8, "stages");
    static_assert(GB == 1 || GB == 2 || GB == 4, "groups per item");
    static_assert(CAP >= kWsListT && CAP % CH == 0, "one round of candidates fits an empty list");
    static constexpr int APlane = 16 * CH * 16;   // one plane (hi or lo) of one group: 2 MN atoms x 2 K groups
    static constexpr int AGroup = 2 * APlane;
    static constexpr int BPlane = 8 * CH * 16;
    static constexpr int StageBytes = GB * AGroup + 2 * BPlane;
    static_assert(StageBytes % 1024 == 0 && APlane % 1024 == 0, "swizzle atoms 1024-byte aligned");
    static constexpr int ListBytes = CAP * 4 + 16 * CAP * 4;   // indices, weights [16][CAP]
    static constexpr size_t Smem = (size_t)NST * StageBytes + 2 * (size_t)ListBytes + 1024;
    static constexpr int AccCols = 64 * GB;                    // one accumulator
    static constexpr int TmemCols = 2 * AccCols;               // two, alternating
    static_assert((GB * CH) % kWsProdWarps == 0, "gather instructions split evenly over the producer warps");
    static_assert(kWsProdT >= CH * 8, "one weight item per producer thread");
};
using WsCfg5 = WsCfg<4, 512, 4>;

template <int NST>
struct WsShared {
    unsigned long long full[NST], empty[NST];   // stage filled (producers: weights, then copies), free (MMA commits)
    unsigned long long lfull[2], lempty[2];     // list segment ready (list warps), consumed (producers)
    unsigned long long afull[2], aempty[2];     // accumulator done (MMA commit), read (epilogue)
    unsigned long long fin;                     // tear-down commit
    unsigned long long never;                   // completed by nobody (the timeout test waits on it)
    int seg_n[2], seg_flags[2];                 // segment: entries; bit 0 first, bit 1 last of the tile
    int st_flags[NST];                          // chunk of a stage: bit 0 first, bit 1 last, ng << 4
    uint32_t tmem;
    int abort;
    int r_beg[kTcMaxRanges], r_pre[kTcMaxRanges + 1], slot_beg[kTcMaxRanges], slot_len[kTcMaxRanges];
    int n_ranges;
};

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// arrive on the barrier once every cp.async this thread has issued so far has
// completed (the barrier's expected count includes this arrival)
__device__ __forceinline__ void mbar_arrive_on_copies(uint32_t mbar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}
// Bounded wait that also returns (false) once another role has set the abort
// flag; a wait that expires sets it.
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort) return false;
        if (clock64() - t0 > kTcWaitCycles) {
            *abort = 1;
            return false;
        }
    }
}
// The same for a whole (converged) warp: one lane waits, the others follow
// it through the shuffle (a warp barrier); the result is warp-uniform.
__device__ __forceinline__ bool ws_wait_warp(uint32_t mbar, uint32_t parity, volatile int *abort) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = ws_wait(mbar, parity, abort);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
// OR of a predicate over the threads of a named barrier (a barrier too; the
// non-aligned forms, so a warp need not arrive converged)
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_named(int id, int nthreads) {
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The work items of one scan (single launch) or of a table of scans (fused
// batch), with the scan's arguments of an item.
struct WsOneScan {
    const GridTcArgs &a;
    int gb;
    __device__ int items() const { return (a.mrx >> 3) * (a.mry >> 3) * ((a.n_g + gb - 1) / gb); }
    __device__ const GridTcArgs &args(int it, int &local) const {
        local = it;
        return a;
    }
    __device__ void mark_timeout() const { atomicOr(&a.hdr->error, kErrTimeout); }
};
struct WsTable {
    const BatchTable<GridTcArgs> &t;
    __device__ int items() const { return t.start[t.n]; }
    __device__ const GridTcArgs &args(int it, int &local) const {
        int lo = 0, hi = t.n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t.start[mid] <= it) lo = mid; else hi = mid;
        }
        local = it - t.start[lo];
        return t.a[lo];
    }
    __device__ void mark_timeout() const {
        for (int i = 0; i < t.n; ++i) atomicOr(&t.a[i].hdr->error, kErrTimeout);
    }
};

// An item's tile and group batch, and whether the tile is live (every role
// walks the same item sequence and skips the same items).  The occupied
// window of the item's scan is read once per scan (it does not change during
// the kernel): most items of a persistent CTA lie outside it.
struct WsItem {
    int tile, g0, ng;
    const WsHeader *hdr = nullptr;   // the scan whose window is cached
    int u_lo = 0, u_len = 0, v_lo = 0, v_len = 0;
};
template <class C>
__device__ __forceinline__ bool ws_item(const GridTcArgs &a, int local, WsItem &w) {
    const int n_tiles = (a.mrx >> 3) * (a.mry >> 3);
    const int gb = local / n_tiles;
    w.tile = local - gb * n_tiles;
    w.g0 = gb * C::GB;
    w.ng = min(C::GB, a.n_g - w.g0);
    if (a.hdr != w.hdr) {
        w.hdr = a.hdr;
        w.u_lo = a.hdr->u_lo;
        w.u_len = a.hdr->u_len;
        w.v_lo = a.hdr->v_lo;
        w.v_len = a.hdr->v_len;
    }
    const int tiles_x = a.mrx >> 3;
    return tile_meets_tc((w.tile % tiles_x) * 8, 8, w.u_lo, w.u_len, a.mrx) &&
           tile_meets_tc((w.tile / tiles_x) * 8, 8, w.v_lo, w.v_len, a.mry);
}

// List warps: the candidate records of each live item's tile, the kept
// samples and their weights, one list segment (at most CAP entries) at a
// time into list buffer (segments published) & 1.
template <class C, class Src>
__device__ __noinline__ void ws_list_role(const Src &src, WsShared<C::NST> &sh, unsigned char *lists) {
    constexpr int CAP = C::CAP;
    const int lt = threadIdx.x - 32 * kWsMmaWarps, lwp = lt >> 5, lane = threadIdx.x & 31;
    __shared__ int wc2[2][kWsListWarps];   // kept per warp, alternating between rounds
    int sc = 0, rnd = 0;
    // the next buffer is free once the producers have issued the segment it
    // held two segments ago (one thread waits, the decision is shared)
    auto acquire = [&]() -> bool {
        bool bad = false;
        if (sc >= 2 && lt == 0) bad = !ws_wait(smem_addr(&sh.lempty[sc & 1]), ((sc >> 1) - 1) & 1, &sh.abort);
        return !bar_or(kWsListBar, kWsListT, bad);
    };
    auto publish = [&](int n, int flags) {
        bar_named(kWsListBar, kWsListT);   // every entry of the segment written
        if (lt == 0) {
            sh.seg_n[sc & 1] = n;
            sh.seg_flags[sc & 1] = flags;
            mbar_arrive(smem_addr(&sh.lfull[sc & 1]));
        }
        ++sc;
    };
    const int items = src.items();
    WsItem w;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        int local;
        const GridTcArgs &a = src.args(it, local);
        if (!ws_item<C>(a, local, w)) continue;
        // stop together once a wait here or in another CTA has expired
        const bool give_up =
            lt == 0 && (*reinterpret_cast<volatile int *>(&sh.abort) ||
                        (*reinterpret_cast<volatile const int *>(&a.hdr->error) & kErrTimeout));
        if (bar_or(kWsListBar, kWsListT, give_up)) {
            if (lt == 0) sh.abort = 1;
            break;
        }
        const int tiles_x = a.mrx >> 3;
        const int U = (w.tile % tiles_x) * 8, V = (w.tile / tiles_x) * 8;
        // candidate bins: first cells u0 in [U - (w - 1), U + 7], v0 likewise;
        // per bin row one or two runs of consecutive bins (two where the run
        // wraps around the periodic grid)
        const int bu_lo = (U - (a.w - 1)) >> 2, bu_hi = (U + 7) >> 2;
        const int bv_lo = (V - (a.w - 1)) >> 2, bv_hi = (V + 7) >> 2;
        if (lt < kTcMaxRanges) {
            const int rr = lt >> 1, part = lt & 1;
            int beg = 0, len = 0;
            if (bv_lo + rr <= bv_hi) {
                const int row = (((bv_lo + rr) % a.nby) + a.nby) % a.nby;
                const int s0 = ((bu_lo % a.nbx) + a.nbx) % a.nbx;
                const int span = bu_hi - bu_lo + 1;
                const int run0 = min(span, a.nbx - s0);
                const int first = part == 0 ? s0 : 0, run = part == 0 ? run0 : span - run0;
                if (run > 0) {
                    beg = a.offsets[row * a.nbx + first];
                    len = a.offsets[row * a.nbx + first + run] - beg;
                }
            }
            sh.slot_beg[lt] = beg;
            sh.slot_len[lt] = len;
        }
        bar_named(kWsListBar, kWsListT);
        if (lt == 0) {
            int n = 0, tot = 0;
            for (int k = 0; k < kTcMaxRanges; ++k)
                if (sh.slot_len[k] > 0) {
                    sh.r_beg[n] = sh.slot_beg[k];
                    sh.r_pre[n] = tot;
                    tot += sh.slot_len[k];
                    ++n;
                }
            sh.r_pre[n] = tot;
            sh.n_ranges = n;
        }
        bar_named(kWsListBar, kWsListT);
        const int n_ranges = sh.n_ranges, total = sh.r_pre[n_ranges];
        const int a_ref = 127 - a.aref[0];
        // the arguments used per candidate, in registers (the barriers are
        // compiler memory barriers: a reference would be re-read after each)
        const int mrx = a.mrx, mry = a.mry, kw = a.w;
        const float kappa = a.kappa;
        const int4 *const trec = a.trec;
        const signed char *const sexp = a.sexp;
        if (!acquire()) break;
        int *lidx = reinterpret_cast<int *>(lists + (sc & 1) * C::ListBytes);
        float *lw = reinterpret_cast<float *>(lidx + CAP);
        auto record = [&](int c) {
            if (c >= total) return make_int4(0, 0, 0, 0);
            int k = 0;
            while (k + 1 < n_ranges && sh.r_pre[k + 1] <= c) ++k;
            return __ldg(trec + sh.r_beg[k] + (c - sh.r_pre[k]));
        };
        int n_list = 0, first = 1;
        bool bad = false;
        // records two rounds ahead, the samples' exponents one round ahead
        // (the exponent load depends on the record: both latencies overlap
        // the rounds instead of adding to them)
        int4 rec_next = record(lt), rec_next2 = record(lt + kWsListT);
        int ex_next = lt < total ? (int)sexp[rec_next.x] : 0;
        for (int base = 0; base < total; base += kWsListT) {
            const int c = base + lt;
            const int4 rec = rec_next;
            const int ex_l = ex_next;
            rec_next = rec_next2;
            ex_next = c + kWsListT < total ? (int)sexp[rec_next.x] : 0;
            rec_next2 = record(c + 2 * kWsListT);
            bool keep = false;
            int l = 0, du = 0, dv = 0;
            float fx = 0.f, fy = 0.f;
            if (c < total) {
                l = rec.x;
                du = (rec.y & 0xffff) - U;
                dv = (rec.y >> 16) - V;
                if (du < -(mrx >> 1)) du += mrx;
                if (du >= (mrx >> 1)) du -= mrx;
                if (dv < -(mry >> 1)) dv += mry;
                if (dv >= (mry >> 1)) dv -= mry;
                fx = __int_as_float(rec.z);
                fy = __int_as_float(rec.w);
                keep = du >= -(kw - 1) && du <= 7 && dv >= -(kw - 1) && dv <= 7;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            int *wc = wc2[rnd & 1];
            ++rnd;
            if (lane == 0) wc[lwp] = __popc(m);
            bar_named(kWsListBar, kWsListT);
            int before = 0, round = 0;
#pragma unroll
            for (int i = 0; i < kWsListWarps; ++i) {
                before += i < lwp ? wc[i] : 0;
                round += wc[i];
            }
            if (n_list + round > CAP) {   // (uniform) the segment is full: hand it over
                publish(n_list, first);
                first = 0;
                n_list = 0;
                if (!acquire()) {
                    bad = true;
                    break;
                }
                lidx = reinterpret_cast<int *>(lists + (sc & 1) * C::ListBytes);
                lw = reinterpret_cast<float *>(lidx + CAP);
            }
            if (keep) {
                const int e = n_list + before + __popc(m & ((1u << lane) - 1u));
                lidx[e] = l;
                // Gaussian weights exp(-kappa (f - tap)^2) on the tile's columns
                // and rows (tap = cell - first cell, zero outside 0 .. w - 1),
                // the rows with the factor 2^(a_ref - a) <= 1 (exact)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int tap = i - du;
                    const float dlt = fx - (float)tap;
                    lw[i * CAP + e] = (tap >= 0 && tap < kw) ? expf(-kappa * dlt * dlt) : 0.f;
                }
                const float scale = ldexpf(1.0f, a_ref - ex_l);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int tap = i - dv;
                    const float dlt = fy - (float)tap;
                    lw[(8 + i) * CAP + e] = (tap >= 0 && tap < kw) ? expf(-kappa * dlt * dlt) * scale : 0.f;
                }
            }
            n_list += round;
        }
        if (bad) break;
        publish(n_list, first | 2);
    }
    __syncwarp();
}

// Producer warps: per chunk of a segment, the split weights and the rows of
// every group of the item (cp.async) into stage k % NST once the MMAs of
// chunk k - NST are done; the stage's barrier completes when every producer
// thread has arrived after its weight stores (with a proxy fence: the tensor
// cores read them) and the copy unit has arrived for each thread's copies.
template <class C, class Src>
__device__ __noinline__ void ws_producer_role(const Src &src, WsShared<C::NST> &sh, unsigned char *stages,
                                              unsigned char *lists) {
    constexpr int CH = C::CH, NST = C::NST, CAP = C::CAP, GB = C::GB;
    const int pt = threadIdx.x - 32 * (kWsMmaWarps + kWsListWarps + kWsEpiWarps), pw = pt >> 5,
              lane = threadIdx.x & 31;
    const uint32_t st0 = smem_addr(stages);
    int sc = 0, k = 0;   // segments consumed, chunks issued
    bool ok = true;
    const int items = src.items();
    WsItem w;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int local;
        const GridTcArgs &a = src.args(it, local);
        if (!ws_item<C>(a, local, w)) continue;
        // the item's row base in registers (not re-read through the argument reference)
        const long long gstride = a.Lmax * 32;
        const uint4 *const shs = a.shs + (long long)w.g0 * gstride;
        bool last = false;
        while (!last) {
            const int b = sc & 1;
            if (!ws_wait_warp(smem_addr(&sh.lfull[b]), (sc >> 1) & 1, &sh.abort)) {
                ok = false;
                break;
            }
            const int n = sh.seg_n[b], fl = sh.seg_flags[b];
            last = (fl & 2) != 0;
            const int *lidx = reinterpret_cast<const int *>(lists + b * C::ListBytes);
            const float *lw = reinterpret_cast<const float *>(lidx + CAP);
            const int nch = n > 0 ? (n + CH - 1) / CH : 1;   // an empty tile: one chunk of zero weights
            for (int q = 0; q < nch; ++q) {
                const int s = k % NST;
                if (k >= NST && !ws_wait_warp(smem_addr(&sh.empty[s]), ((k / NST) - 1) & 1, &sh.abort)) {
                    ok = false;
                    break;
                }
                const int base = q * CH;
                unsigned char *st = stages + s * C::StageBytes;
                // split weights: one (sample, cell row) item of 8 cells per thread
                if (pt < CH * 8) {
                    const int j = pt % CH, rrow = pt / CH;
                    const int e = base + j;
                    float v[8];
                    const float wy = e < n ? lw[(8 + rrow) * CAP + e] : 0.f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = e < n ? lw[i * CAP + e] * wy : 0.f;
                    uint4 hi, lo;
                    split8(v, hi, lo);
                    unsigned char *d = st + GB * C::AGroup + rrow * (CH * 16) + j * 16;
                    *reinterpret_cast<uint4 *>(d) = hi;
                    *reinterpret_cast<uint4 *>(d + C::BPlane) = lo;
                }
                if (pt == 0)
                    sh.st_flags[s] = (((fl & 1) && q == 0) ? 1 : 0) | ((last && q == nch - 1) ? 2 : 0) | (w.ng << 4);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_addr(&sh.full[s]));   // weights and chunk flags written

                // rows: per group and plane the two 128-byte halves of each of
                // the CH samples, one warp-instruction per 4 samples x 128
                // bytes (whole lines); stored in the 128-byte-swizzled
                // MN-major layout of the A operands: 16-byte chunk c of sample
                // j's half h at h * 2048 + (j / 8) * 1024 + (j % 8) * 128 +
                // (c ^ j % 8) * 16 (an atom is 8 samples x 64 halves)
                constexpr int NR = GB * 16 / kWsProdWarps;
                int lr[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {   // the listed samples first (independent loads)
                    const int i = pw + kWsProdWarps * r;
                    const int e = base + 4 * (i & 3) + (lane >> 3);
                    lr[r] = e < n ? lidx[e] : 0;
                }
                const uint32_t sst = st0 + s * C::StageBytes;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int i = pw + kWsProdWarps * r;   // (group, plane, half, sample quad)
                    const int gl = i >> 4, plane = (i >> 3) & 1, h = (i >> 2) & 1, sq = i & 3;
                    if (gl >= w.ng) continue;
                    const int j = 4 * sq + (lane >> 3), c = lane & 7;
                    const uint4 *srcp = shs + gl * gstride + (long long)lr[r] * 32 + plane * 16 + 8 * h + c;
                    cp_async16_free(sst + gl * C::AGroup + plane * C::APlane + h * 2048 + (j >> 3) * 1024 +
                                        (j & 7) * 128 + ((c ^ (j & 7)) << 4),
                                    srcp);
                }
                mbar_arrive_on_copies(smem_addr(&sh.full[s]));   // the copies, once landed
                ++k;
            }
            if (!ok) break;
            mbar_arrive(smem_addr(&sh.lempty[b]));   // the segment's entries are no longer read
            ++sc;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // no copy of this thread outlives the kernel
    __syncwarp();
}

// MMA warps (one thread each; warp mw takes groups mw, mw + kWsMmaWarps, ...):
// per chunk, three MMAs per group into the item's accumulator (the first
// chunk of a tile overwrites it), the stage committed back to the producers;
// after a tile's last chunk the accumulator is committed to the epilogue.
// Accumulator t % 2 is reused by tile t once the epilogue has read tile t - 2
// from it.  (Two issuing threads: an MMA instruction occupies its thread for
// longer than the tensor pipe needs to execute it.)
template <class C, class Src>
__device__ __noinline__ void ws_mma_role(const Src &src, WsShared<C::NST> &sh, unsigned char *stages, int mw) {
    constexpr int NST = C::NST, GB = C::GB;
    static_assert(C::CH == 16, "one K step per chunk");
    // stage 0's operand descriptors: A with the 128-byte swizzle (MN atoms 2048
    // bytes apart, 8-sample groups 1024 apart), B without (core matrices of 8
    // samples x 16 bytes, K-adjacent 128 bytes apart, MN-adjacent 256)
    const uint64_t da0 = tc_desc_sw128(smem_addr(stages), 2048, 1024);
    const uint64_t db0 = tc_desc(smem_addr(stages) + GB * C::AGroup, 128, C::CH * 16);
    int k = 0, tcount = 0;
    const int items = src.items();
    WsItem w;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        int local;
        const GridTcArgs &a = src.args(it, local);
        if (!ws_item<C>(a, local, w)) continue;
        const int ab = tcount & 1;
        // the timeout test: a wait that runs out, as a lost arrival would make it
        if (a.wait_test && mw == 0 && !ws_wait(smem_addr(&sh.never), 0, &sh.abort)) break;
        if (tcount >= 2 && !ws_wait(smem_addr(&sh.aempty[ab]), ((tcount >> 1) - 1) & 1, &sh.abort)) break;
        const uint32_t acc = sh.tmem + (uint32_t)(ab * C::AccCols);
        bool ok = true, tile_done = false;
        while (!tile_done) {
            const int s = k % NST;
            if (!ws_wait(smem_addr(&sh.full[s]), (k / NST) & 1, &sh.abort)) {
                ok = false;
                break;
            }
            // the producers' copies landed through the generic proxy: make them
            // visible to the tensor cores' (async proxy) reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int fl = sh.st_flags[s], ng = fl >> 4;
            // descriptors of this stage: those of stage 0 plus the byte offset / 16
            // (the 14-bit address field cannot carry: shared addresses < 256 KB)
            const uint64_t so = (uint64_t)((s * C::StageBytes) >> 4);
            const uint64_t dbh = db0 + so, dbl = dbh + (C::BPlane >> 4);
#pragma unroll
            for (int gl = mw; gl < GB; gl += kWsMmaWarps) {
                if (gl >= ng) break;
                const uint64_t dah = da0 + so + (uint64_t)((gl * C::AGroup) >> 4), dal = dah + (C::APlane >> 4);
                const uint32_t d = acc + 64u * gl;
                tc_mma(d, dah, dbh, (fl & 1) ? 0u : 1u);
                tc_mma(d, dah, dbl, 1u);
                tc_mma(d, dal, dbh, 1u);
            }
            tc_commit(smem_addr(&sh.empty[s]));
            ++k;
            if (fl & 2) {
                tc_commit(smem_addr(&sh.afull[ab]));
                tile_done = true;
            }
        }
        if (!ok) break;
        ++tcount;
    }
    // every MMA issued has completed before the stages and tensor memory go
    tc_commit(smem_addr(&sh.fin));
    if (!mbar_wait_bounded(smem_addr(&sh.fin), 0)) sh.abort = 1;
}

// Epilogue warps: lane quarter warp % 4 of each accumulator, x 2^-a_ref, to G
// (row m = 32 (warp % 4) + lane: frequency 64 g + m / 2, component m % 2;
// column n: cell (U + n % 8, V + n / 8)).
template <class C, class Src>
__device__ __noinline__ void ws_epilogue_role(const Src &src, WsShared<C::NST> &sh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, mrow = 32 * quarter + lane;
    int tcount = 0;
    const int items = src.items();
    WsItem w;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        int local;
        const GridTcArgs &a = src.args(it, local);
        if (!ws_item<C>(a, local, w)) continue;
        const int ab = tcount & 1;
        if (!ws_wait_warp(smem_addr(&sh.afull[ab]), (tcount >> 1) & 1, &sh.abort)) break;   // (warp-uniform)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int tiles_x = a.mrx >> 3;
        const int U = (w.tile % tiles_x) * 8, V = (w.tile / tiles_x) * 8;
        const float unscale = ldexpf(1.0f, -(127 - a.aref[0]));
        const int mrx = a.mrx, n_kc = a.n_kc;
        const long long plane_stride = (long long)a.mry * a.mrx * kKC;
        float2 *const G = a.G;
        const uint32_t tmem = sh.tmem;
        for (int gl = 0; gl < w.ng; ++gl) {
            const int f = 64 * (w.g0 + gl) + (mrow >> 1);
            const int kc = f >> 5;
            const bool live = kc < n_kc;
            // cell (U, V) of this row's frequency plane; cell (U + col, V + row)
            // is row x rstride + col x 64 floats further
            float *const cell0 = live ? reinterpret_cast<float *>(G + (long long)kc * plane_stride) + 2 * (f & 31) +
                                            (mrow & 1) + ((long long)V * mrx + U) * (2 * kKC)
                                      : nullptr;
            const long long rstride = (long long)mrx * (2 * kKC);
#pragma unroll 1
            for (int c0 = 0; c0 < 64; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) +
                                       (uint32_t)(ab * C::AccCols + 64 * gl + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n\ttcgen05.wait::ld.sync.aligned;"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
                if (live) {
                    float *const row0 = cell0 + (c0 >> 3) * rstride;   // columns c0 .. c0 + 15: two cell rows
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        row0[(i >> 3) * rstride + (i & 7) * (2 * kKC)] = __uint_as_float(r[i]) * unscale;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&sh.aempty[ab]));
        ++tcount;
    }
    __syncwarp();
}

template <class C, class Src>
__device__ __forceinline__ void grid_ws_body(const Src &src, unsigned char *smem, WsShared<C::NST> &sh) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < C::NST; ++s) {
            mbar_init(smem_addr(&sh.full[s]), 2 * kWsProdT);   // weights + copies per producer thread
            mbar_init(smem_addr(&sh.empty[s]), kWsMmaWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_addr(&sh.lfull[b]), 1);
            mbar_init(smem_addr(&sh.lempty[b]), kWsProdT);
            mbar_init(smem_addr(&sh.afull[b]), kWsMmaWarps);
            mbar_init(smem_addr(&sh.aempty[b]), kWsEpiWarps);
        }
        mbar_init(smem_addr(&sh.fin), kWsMmaWarps);
        mbar_init(smem_addr(&sh.never), 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sh.tmem)),
                     "r"(C::TmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    unsigned char *stages = smem, *lists = smem + C::NST * C::StageBytes;
    if (warp < kWsMmaWarps) {
        if (lane == 0) ws_mma_role<C>(src, sh, stages, warp);
        __syncwarp();
    } else if (warp < kWsMmaWarps + kWsListWarps) {
        ws_list_role<C>(src, sh, lists);
    } else if (warp < kWsMmaWarps + kWsListWarps + kWsEpiWarps) {
        ws_epilogue_role<C>(src, sh);
    } else {
        ws_producer_role<C>(src, sh, stages, lists);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *reinterpret_cast<volatile int *>(&sh.abort)) src.mark_timeout();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(C::TmemCols));
    }
}

template <class C>
__global__ void __launch_bounds__(kWsT, 1) grid_ws_kernel(const __grid_constant__ GridTcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) WsShared<C::NST> sh;
    grid_ws_body<C>(WsOneScan{a, C::GB}, smem, sh);
}

template <class C>
__global__ void __launch_bounds__(kWsT, 1) grid_ws_multi(const __grid_constant__ BatchTable<GridTcArgs> t) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) WsShared<C::NST> sh;
    grid_ws_body<C>(WsTable{t}, smem, sh);
}

static int grid_tc_describe(const Plan &p, void *ws, GridTcArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.shs = reinterpret_cast<const uint4 *>(w + p.off_shat);
    a.sexp = reinterpret_cast<const signed char *>(w + p.off_sexp);
    a.aref = reinterpret_cast<const int *>(w + p.off_aref);
    a.trec = reinterpret_cast<const int4 *>(w + p.off_trec);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.G = reinterpret_cast<float2 *>(w + p.off_G);
    a.hdr = reinterpret_cast<WsHeader *>(w);
    a.Lmax = p.L;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.nby = p.nby;
    a.w = p.w;
    a.n_kc = p.n_kc;
    a.n_g = (p.n_kc + 1) / 2;
    a.kappa = (float)(1.5 * kPi / p.w);
    a.wait_test = p.wait_test;
    return (p.mrx / 8) * (p.mry / 8);   // tiles
}

// work items of a scan for a variant: tiles x group batches
static int tc_items(int tiles, const GridTcArgs &a, int gb) { return tiles * ((a.n_g + gb - 1) / gb); }

// CTAs of a persistent launch: MINB per SM (the shared-memory limit)
static int tc_persistent_ctas(int items, int minb) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            sms = n;
        else
            sms = 148;
    }
    return std::max(1, std::min(items, minb * sms));
}

template <class C>
static cudaError_t grid_tc_launch(const GridTcArgs *a, const BatchTable<GridTcArgs> *t, int items, cudaStream_t s) {
    if (a) {
        cudaError_t e = ensure_smem_attr((const void *)grid_tc_kernel<C>, C::Smem);
        if (e != cudaSuccess) return e;
        grid_tc_kernel<C><<<tc_persistent_ctas(items, C::MINB), C::T, C::Smem, s>>>(*a);
    } else {
        cudaError_t e = ensure_smem_attr((const void *)grid_tc_multi<C>, C::Smem);
        if (e != cudaSuccess) return e;
        grid_tc_multi<C><<<tc_persistent_ctas(items, C::MINB), C::T, C::Smem, s>>>(*t);
    }
    return cudaGetLastError();
}

template <class C>
static cudaError_t grid_ws_launch(const GridTcArgs *a, const BatchTable<GridTcArgs> *t, int items, cudaStream_t s) {
    // one CTA per SM (its shared memory and tensor memory take the SM)
    if (a) {
        cudaError_t e = ensure_smem_attr((const void *)grid_ws_kernel<C>, C::Smem);
        if (e != cudaSuccess) return e;
        grid_ws_kernel<C><<<tc_persistent_ctas(items, 1), kWsT, C::Smem, s>>>(*a);
    } else {
        cudaError_t e = ensure_smem_attr((const void *)grid_ws_multi<C>, C::Smem);
        if (e != cudaSuccess) return e;
        grid_ws_multi<C><<<tc_persistent_ctas(items, 1), kWsT, C::Smem, s>>>(*t);
    }
    return cudaGetLastError();
}

static int tc_variant_gb(int variant) {
    switch (variant) {
        case 5: return WsCfg5::GB;
        case 1: return TcCfg1::GB;
        case 3: return TcCfg3::GB;
        case 4: return TcCfg4::GB;
        default: return TcCfg2::GB;
    }
}

static cudaError_t grid_tc_dispatch(int variant, const GridTcArgs *a, const BatchTable<GridTcArgs> *t, int items,
                                    cudaStream_t s) {
    switch (variant) {
        case 5: return grid_ws_launch<WsCfg5>(a, t, items, s);
        case 1: return grid_tc_launch<TcCfg1>(a, t, items, s);
        case 3: return grid_tc_launch<TcCfg3>(a, t, items, s);
        case 4: return grid_tc_launch<TcCfg4>(a, t, items, s);
        default: return grid_tc_launch<TcCfg2>(a, t, items, s);
    }
}

cudaError_t launch_grid_tc(const Plan &p, void *ws, cudaStream_t s) {
    GridTcArgs a;
    const int tiles = grid_tc_describe(p, ws, a);
    return grid_tc_dispatch(p.tc, &a, nullptr, tc_items(tiles, a, tc_variant_gb(p.tc)), s);
}

cudaError_t launch_grid_tc_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<GridTcArgs> args((size_t)n);
    std::vector<int> blocks((size_t)n), keys((size_t)n, 0);
    bool any = false;
    for (int i = 0; i < n; ++i) {
        const int v = r[i].plan->p.tc;
        const int tiles = grid_tc_describe(r[i].plan->p, r[i].workspace, args[i]);
        blocks[i] = v ? tc_items(tiles, args[i], tc_variant_gb(v)) : 0;   // other plans: the FP32 forms
        keys[i] = v;                                                       // one fused launch per variant
        any |= blocks[i] > 0;
    }
    if (!any) return cudaSuccess;
    return launch_groups(n, keys.data(), args.data(), blocks.data(),
                         [&](int key, const BatchTable<GridTcArgs> &t, int total) {
                             return grid_tc_dispatch(key, nullptr, &t, total, s);
                         });
}

}  // namespace mmsar
