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

static int tc_variant_gb(int variant) {
    switch (variant) {
        case 1: return TcCfg1::GB;
        case 3: return TcCfg3::GB;
        case 4: return TcCfg4::GB;
        default: return TcCfg2::GB;
    }
}

static cudaError_t grid_tc_dispatch(int variant, const GridTcArgs *a, const BatchTable<GridTcArgs> *t, int items,
                                    cudaStream_t s) {
    switch (variant) {
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
