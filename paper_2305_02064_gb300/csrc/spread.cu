// Gaussian gridding (the spreading step of the fast Gaussian gridding NUFFT
// that Sec. III uses for FT_2D of Eq. 16) of the compensated virtual-array
// samples onto the 2Mx x 2My periodic aperture grid, in gather form.
//
// Weight of a sample at grid position g for cell j: exp(-kappa (g - j)^2)
// with kappa = h^2 / (4 tau) = 1.5 pi / w for the Greengard-Lee tau and a
// cell size h = 2 pi / (2M); the sample reaches the w cells
// u0 .. u0 + w - 1, u0 = ceil(g - w/2) (indices modulo the grid size).
//
// The per-sample records it reads (bin order; written with the in-bin sort,
// see samples.cu): the sample's offset inside its 4x4-cell bin and original
// index, and per axis w + 3 "quads" -- quad q holds the weights of taps
// q-3 .. q (zero outside 0..w-1), i.e. exactly the four weights a 4-cell
// block needs when it starts q - 3 cells after u0.  The compensated samples
// are in original sample order.
//
// spread_kernel: a CTA owns a tile of grid cells and a group of frequency
// chunks; each of its warps owns a block of cells (4 x 4, or 4 x 2 when a lane
// keeps four frequencies), and each lane keeps in registers the complex
// accumulators of its frequencies over the block.  Warps work independently
// (no block barrier): a warp walks the bins whose samples can reach its block,
// tests 32 samples at a time (one lane each) for overlap with the block and
// appends the overlapping ones to a list in shared memory -- the sample index
// and, gathered from the records, the two weight quads its position in the
// block selects -- then applies the list with the compensated values of the
// next few entries in flight.  For a bin d bins before the block, the block
// starts 4 d - (in-bin offset) cells after the sample's first tap (plus the
// block's own offset inside its bin), which selects one weight quad per axis.
// No two warps write the same cell: no atomics, a fixed summation order, the
// same for every launch shape (so all shapes give the same bits).
#include "fft.cuh"
#include "internal.cuh"

namespace mmsar {

struct SpreadArgs {
    const float2 *shat;       // [n_kc / 2][Lmax][64], original sample order
    const int2 *dd;           // [Lmax] (in-bin offset du | dv << 2, sample index), bin order
    const float4 *wrec;       // [Lmax][2 (w + 3) + 1]: header + x quads + y quads
    const int *offsets;       // [n_bins + 1]
    float2 *G;                // [n_kc][mry][mrx][32]
    const WsHeader *hdr;      // occupied window of the grid
    long long Lmax;
    int mrx, mry, nbx, nby;
    int w, nb, n_kc;          // taps per axis; bins visited per axis; frequency chunks
};

// Does [t0, t0 + span) meet the periodic window lo .. lo + len - 1 (mod m)?
__device__ __forceinline__ bool tile_meets(int t0, int span, int lo, int len, int m) {
    if (len >= m) return true;
    if (len <= 0) return false;
    int d = (t0 - lo) % m;
    if (d < 0) d += m;
    int e = (lo - t0) % m;
    if (e < 0) e += m;
    return d < len || e < span;
}

constexpr int kListCap = 192;   // relevant samples listed per warp before they are applied

// NF: frequencies per lane (1: a CTA covers one chunk of 32 frequencies; 2:
// a 64-frequency group, lane l holding frequencies 2l and 2l + 1; 4: a
// 128-frequency group, lane l holding 4l .. 4l + 3); WARPS: 4 or 8, in two
// block rows.  Warp blocks are 4 x 4 cells, or 4 x 2 for NF = 4 (the same
// accumulator count per lane; fewer taps outside the sample's support:
// (w + 3)(w + 1) cells visited per sample instead of (w + 3)^2).
template <int NF, int WARPS, int NS, int MINB>
__device__ __forceinline__ void spread_body(const SpreadArgs &a, int bid) {
    constexpr int BY = NF == 4 ? 2 : 4;   // block rows (cells along y')
    constexpr int TX = 4 * (WARPS / 2);   // tile width in cells (two block rows)
    constexpr int TY = 2 * BY;
    // per warp and listed sample: its x and y weight quads (gathered from the
    // records while the list is built, one lane per sample) and its index;
    // eight warps list fewer samples at a time (static shared memory <= 48 KB)
    constexpr int CAP = WARPS == 8 ? 160 : kListCap;
    __shared__ float4 lquads[WARPS][CAP][2];
    __shared__ int lidx[WARPS][CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = a.mrx / TX;
    // the frequency group varies fastest, so the groups of one tile run
    // together and share its weight records in L2
    const int n_kg = (a.n_kc + NF - 1) / NF;
    const int kg = bid % n_kg;
    const int tile = bid / n_kg;
    // tiles outside the occupied window stay unwritten: the FFT along x'
    // reads only the window and takes the rest as zero
    if (!tile_meets((tile % tiles_x) * TX, TX, a.hdr->u_lo, a.hdr->u_len, a.mrx) ||
        !tile_meets((tile / tiles_x) * TY, TY, a.hdr->v_lo, a.hdr->v_len, a.mry))
        return;
    const int U = (tile % tiles_x) * TX + (warp % (WARPS / 2)) * 4;
    const int V = (tile / tiles_x) * TY + (warp / (WARPS / 2)) * BY;
    const int rq = 2 * (a.w + 3) + 1;
    const int nq = a.w + 3;
    float2 acc[NF][BY][4];   // (re, im) per frequency of the lane and cell
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int j = 0; j < BY; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[f][j][i] = make_float2(0.f, 0.f);
    // s_hat: [(n_kc + 1) / 2][Lmax][64] complex; the lane's NF values of a
    // sample are 8 NF contiguous bytes at row offset (sample * 64 + col0)
    // complex of 64-frequency group gi (for NF = 4 the upper half-warp reads
    // the second group, absent when the chunk count leaves it out)
    const int gi = NF == 4 ? 2 * kg + (lane >> 4) : NF == 2 ? kg : kg >> 1;
    const int col0 = NF == 4 ? 4 * (lane & 15) : NF == 2 ? 2 * lane : (kg & 1) * 32 + lane;
    const bool has = NF != 4 || gi < (a.n_kc + 1) / 2;
    const float2 *sh = a.shat + (long long)(has ? gi : 0) * a.Lmax * 64 + col0;
    float4 (*quads)[2] = lquads[warp];
    int *sidx = lidx[warp];

    // one listed sample in flight: its values (the weights wait in shared memory)
    struct Stage {
        float2 v[NF];
    };
    // apply the listed samples through an NS-deep pipeline: the loads of
    // entry i + NS are issued as soon as entry i has been accumulated
    auto apply = [&](int n) {
        Stage st[NS];
        auto fetch = [&](int i, Stage &q) {
            const int l = sidx[i];
            if constexpr (NF == 4) {
                // sample index * 32 < 2^31 (plan limit): 32-bit offsets in float4 units
                float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = t0;
                if (has) {
                    const float4 *p4 = reinterpret_cast<const float4 *>(sh) + (l << 5);
                    t0 = __ldg(p4);
                    t1 = __ldg(p4 + 1);
                }
                q.v[0] = make_float2(t0.x, t0.y);
                q.v[1] = make_float2(t0.z, t0.w);
                q.v[2] = make_float2(t1.x, t1.y);
                q.v[NF - 1] = make_float2(t1.z, t1.w);
            } else if constexpr (NF == 2) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(sh) + (l << 5));
                q.v[0] = make_float2(t.x, t.y);
                q.v[NF - 1] = make_float2(t.z, t.w);
            } else {
                q.v[0] = __ldg(sh + ((long long)l << 6));
            }
        };
        auto consume = [&](int i, const Stage &q) {
            const float4 qx = quads[i][0], qy = quads[i][1];
            const float wx[4] = {qx.x, qx.y, qx.z, qx.w};
            const float wy[4] = {qy.x, qy.y, qy.z, qy.w};
            // (re, im) pairs in packed two-lane FP32 instructions
#pragma unroll
            for (int j = 0; j < BY; ++j) {
                const float2 wyj = make_float2(wy[j], wy[j]);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const float2 t = fmul2(wyj, q.v[f]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[f][j][i] = ffma2(make_float2(wx[i], wx[i]), t, acc[f][j][i]);
                }
            }
        };
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if (k < n) fetch(k, st[k]);
        for (int i = 0; i < n; i += NS) {
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                if (i + k >= n) break;
                consume(i + k, st[k]);
                if (i + k + NS < n) fetch(i + k + NS, st[k]);
            }
        }
    };

    const int bu0 = U >> 2, bv0 = V >> 2;
    const int v_in = V & 3;   // the block's first row inside its bin (0, or 2 for 4 x 2 blocks)
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int dbv = a.nb - 1; dbv >= 0; --dbv) {
        int bv = bv0 - dbv;
        if (bv < 0) bv += a.nby;
        for (int dbu = a.nb - 1; dbu >= 0; --dbu) {
            int bu = bu0 - dbu;
            if (bu < 0) bu += a.nbx;
            const int bin = bv * a.nbx + bu;
            const int beg = __ldg(a.offsets + bin), end = __ldg(a.offsets + bin + 1);
            for (int s0 = beg; s0 < end; s0 += 32) {
                // which of the next 32 samples reach this block, in one step
                const int my = s0 + lane;
                bool rel = false;
                int4 ent = make_int4(0, 0, 0, 0);
                if (my < end) {
                    const int2 ds = __ldg(a.dd + my);
                    const int d = ds.x;
                    const int ru = 4 * dbu - (d & 3);             // block start relative to the first tap, >= -3
                    const int rv = 4 * dbv - (d >> 2) + v_in;     // >= -3; a 4 x 2 block needs >= -1
                    rel = ru < a.w && rv < a.w && rv > -BY;
                    const int base = my * rq + 1;                 // the sample's x quads, then its y quads
                    ent = make_int4(base + ru + 3, base + nq + rv + 3, ds.y, 0);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, rel);
                if (n + __popc(mask) > CAP) {   // keep the list within its buffer
                    __syncwarp();
                    apply(n);
                    n = 0;
                    __syncwarp();
                }
                if (rel) {
                    const int pos = n + __popc(mask & lt);
                    quads[pos][0] = __ldg(a.wrec + ent.x);
                    quads[pos][1] = __ldg(a.wrec + ent.y);
                    sidx[pos] = ent.z;
                }
                n += __popc(mask);
            }
        }
    }
    __syncwarp();
    apply(n);
    if constexpr (NF == 4) {
        // lane l holds chunk 4 kg + l / 8 (absent past the chunk count),
        // complex 4 (l % 8) .. + 3 of it: 32 bytes per lane, 256 contiguous bytes per chunk
        const int kc = 4 * kg + (lane >> 3);
        if (kc < a.n_kc) {
            float4 *g = reinterpret_cast<float4 *>(a.G + (long long)kc * a.mry * a.mrx * kKC) + 2 * (lane & 7);
#pragma unroll
            for (int j = 0; j < BY; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float4 *c = g + ((long long)(V + j) * a.mrx + (U + i)) * (kKC / 2);
                    c[0] = make_float4(acc[0][j][i].x, acc[0][j][i].y, acc[1][j][i].x, acc[1][j][i].y);
                    c[1] = make_float4(acc[2][j][i].x, acc[2][j][i].y, acc[NF - 1][j][i].x, acc[NF - 1][j][i].y);
                }
        }
    } else if constexpr (NF == 2) {
        // lanes 0..15 hold chunk 2 kg, lanes 16..31 chunk 2 kg + 1 (absent when
        // the chunk count is odd): 16 bytes per lane, 256 contiguous bytes per chunk
        const int kc = 2 * kg + (lane >> 4);
        if (kc < a.n_kc) {
            float4 *g = reinterpret_cast<float4 *>(a.G + (long long)kc * a.mry * a.mrx * kKC) + (lane & 15);
#pragma unroll
            for (int j = 0; j < BY; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    g[((long long)(V + j) * a.mrx + (U + i)) * (kKC / 2)] =
                        make_float4(acc[0][j][i].x, acc[0][j][i].y, acc[NF - 1][j][i].x, acc[NF - 1][j][i].y);
        }
    } else {
        float2 *g = a.G + (long long)kg * a.mry * a.mrx * kKC + lane;
#pragma unroll
        for (int j = 0; j < BY; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) g[((long long)(V + j) * a.mrx + (U + i)) * kKC] = acc[0][j][i];
    }
}

template <int NF, int WARPS, int NS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) spread_kernel(const SpreadArgs a) {
    spread_body<NF, WARPS, NS, MINB>(a, blockIdx.x);
}

template <int NF, int WARPS, int NS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) spread_multi(const __grid_constant__ BatchTable<SpreadArgs> t) {
    __shared__ SpreadArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    spread_body<NF, WARPS, NS, MINB>(sa, bid);
}

static int spread_describe(const Plan &p, void *ws, SpreadArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.shat = reinterpret_cast<const float2 *>(w + p.off_shat);
    a.dd = reinterpret_cast<const int2 *>(w + p.off_dd);
    a.wrec = reinterpret_cast<const float4 *>(w + p.off_wq);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.G = reinterpret_cast<float2 *>(w + p.off_G);
    a.hdr = reinterpret_cast<const WsHeader *>(w);
    a.Lmax = p.L;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.nby = p.nby;
    a.w = p.w;
    a.nb = (p.w - 1 + kBin - 1) / kBin + 1;
    a.n_kc = p.n_kc;
    const int nf = p.spread_nf, warps = p.spread_warps;
    const int tiles = (p.mrx / (2 * warps)) * (p.mry / (nf == 4 ? 4 : 8));
    return tiles * ((p.n_kc + nf - 1) / nf);
}

template <int NF, int WARPS, int NS, int MINB>
static void spread_launch(const SpreadArgs *a, const BatchTable<SpreadArgs> *t, int blocks, cudaStream_t s) {
    if (a)
        spread_kernel<NF, WARPS, NS, MINB><<<blocks, WARPS * 32, 0, s>>>(*a);
    else
        spread_multi<NF, WARPS, NS, MINB><<<blocks, WARPS * 32, 0, s>>>(*t);
}

// key: 2 x frequencies per lane + (8 warps)
static void spread_dispatch(int key, const SpreadArgs *a, const BatchTable<SpreadArgs> *t, int blocks,
                            cudaStream_t s) {
    switch (key) {
        case 9: spread_launch<4, 8, 4, 2>(a, t, blocks, s); break;
        case 8: spread_launch<4, 4, 4, 4>(a, t, blocks, s); break;
        case 5: spread_launch<2, 8, 8, 2>(a, t, blocks, s); break;
        case 4: spread_launch<2, 4, 8, 4>(a, t, blocks, s); break;
        case 3: spread_launch<1, 8, 8, 2>(a, t, blocks, s); break;
        default: spread_launch<1, 4, 8, 5>(a, t, blocks, s); break;
    }
}

cudaError_t launch_spread(const Plan &p, void *ws, cudaStream_t s) {
    // the launch shape is the plan's (set by mmsar_plan_set_tiles, e.g. from
    // the autotuner): NF frequencies per lane, WARPS warps per CTA; 32 bytes
    // of compensated values per lane in flight (eight listed samples, four
    // for NF = 4; the weights wait in the shared-memory list)
    SpreadArgs a;
    const int blocks = spread_describe(p, ws, a);
    spread_dispatch(2 * p.spread_nf + (p.spread_warps == 8 ? 1 : 0), &a, nullptr, blocks, s);
    return cudaGetLastError();
}

}  // namespace mmsar

// ---------------------------------------------------------------- grouped gridding
// The samples of one position whose Tx/Rx pairs share the x offset (the same
// x', Eq. 3) share the x weights, so a warp block sums such a group's
// samples into one y-weighted value per block row first,
//     T_j = sum_e wy_j(e) s_hat_e,
// and applies the x weights once per group: acc_ji += wx_i T_j (for the
// 4 x 4 block, 8 multiply-adds per sample and 16 per group, instead of 16 per
// sample).  The bins hold groups (by their x cell and their lowest first y
// cell); a warp tests 32 groups at a time, one lane each, lists the group's
// samples that reach its rows next to each other (the last one flagged), and
// applies the list through the same pipeline as the per-sample kernel.
namespace mmsar {

struct SpreadGroupArgs {
    const float2 *shat;       // [n_kc / 2][Lmax][64], original sample order
    const int2 *gdd;          // [G] per sorted group: (du | dv << 2 of its lowest first cell, group)
    const float4 *gxq;        // [G][w + 3] x quads per sorted group
    const float4 *yq;         // [Lmax][w + 4] per sample: offset header, y quads
    const int4 *goff;         // [G][2] per sorted group: members' y offsets, uint16 x 16
    const int *offsets;       // [n_bins + 1] group bins
    const int *cls;           // pair classes, class starts, members
    float2 *G;
    const WsHeader *hdr;
    long long Lmax;
    int P, TR;
    int mrx, mry, nbx, nby;
    int w, nb, n_kc;
};

template <int NF, int WARPS, int NS, int MINB>
__device__ __forceinline__ void spread_groups_body(const SpreadGroupArgs &a, int bid) {
    constexpr int TX = 4 * (WARPS / 2);
    // per warp: (x-quad index, y-quad index, sample index, last of its group)
    __shared__ int4 lists[WARPS][kListCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = a.mrx / TX;
    const int n_kg = NF == 2 ? (a.n_kc + 1) / 2 : a.n_kc;
    const int kg = bid % n_kg;
    const int tile = bid / n_kg;
    if (!tile_meets((tile % tiles_x) * TX, TX, a.hdr->u_lo, a.hdr->u_len, a.mrx) ||
        !tile_meets((tile / tiles_x) * 8, 8, a.hdr->v_lo, a.hdr->v_len, a.mry))
        return;
    const int U = (tile % tiles_x) * TX + (warp % (WARPS / 2)) * 4;
    const int V = (tile / tiles_x) * 8 + (warp / (WARPS / 2)) * 4;
    const int nqx = a.w + 3, rqy = a.w + 4;
    const int vspan = a.hdr->vspan_max;
    // bin rows of a group's lowest first y cell that can reach the block rows
    const int nbv = min((vspan + a.w + 2) / 4 + 1, a.nby);
    // the class tables in shared memory: class starts, then members
    __shared__ int ctab[2 * kMaxPairsGrouped + 1];
    for (int i = threadIdx.x; i < 2 * a.TR + 1; i += blockDim.x) ctab[i] = a.cls[a.TR + i];
    __syncthreads();
    const int *cstart = ctab, *members = ctab + a.TR + 1;
    float2 acc[NF][4][4];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[f][j][i] = make_float2(0.f, 0.f);
    const int col0 = NF == 2 ? 2 * lane : (kg & 1) * 32 + lane;
    const float2 *sh = a.shat + (long long)(NF == 2 ? kg : kg >> 1) * a.Lmax * 64 + col0;
    int4 *list = lists[warp];

    struct Stage {
        float4 x, y;
        float2 v[NF];
        int last;
    };
    auto apply = [&](int n) {
        float2 T[NF][4];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int j = 0; j < 4; ++j) T[f][j] = make_float2(0.f, 0.f);
        Stage st[NS];
        auto fetch = [&](int i, Stage &q) {
            const int4 e = list[i];
            q.x = __ldg(a.gxq + e.x);
            q.y = __ldg(a.yq + e.y);
            q.last = e.w;
            if constexpr (NF == 2) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(sh) + (e.z << 5));
                q.v[0] = make_float2(t.x, t.y);
                q.v[NF - 1] = make_float2(t.z, t.w);
            } else {
                q.v[0] = __ldg(sh + ((long long)e.z << 6));
            }
        };
        auto consume = [&](const Stage &q) {
            const float wy[4] = {q.y.x, q.y.y, q.y.z, q.y.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 wyj = make_float2(wy[j], wy[j]);
#pragma unroll
                for (int f = 0; f < NF; ++f) T[f][j] = ffma2(wyj, q.v[f], T[f][j]);
            }
            if (q.last) {   // the group is complete: its x weights, once
                const float wx[4] = {q.x.x, q.x.y, q.x.z, q.x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 wxi = make_float2(wx[i], wx[i]);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int f = 0; f < NF; ++f) acc[f][j][i] = ffma2(wxi, T[f][j], acc[f][j][i]);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int j = 0; j < 4; ++j) T[f][j] = make_float2(0.f, 0.f);
            }
        };
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if (k < n) fetch(k, st[k]);
        for (int i = 0; i < n; i += NS) {
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                if (i + k >= n) break;
                consume(st[k]);
                if (i + k + NS < n) fetch(i + k + NS, st[k]);
            }
        }
    };

    // the candidate groups of all nbv x nb bins around the block, enumerated as
    // one sequence (bin by bin, in bin order) so that every 32-lane round is
    // full: lane b < nbins holds bin b's start and its first index in the
    // sequence.  Bins are visited in chunks of 32.
    const int bu0 = U >> 2, bv0 = V >> 2;
    const int nbins = nbv * a.nb;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int b0 = 0; b0 < nbins; b0 += 32) {
        int beg = 0, cnt_b = 0, dbu = 0, dbv = 0;
        const int b = b0 + lane;
        if (b < nbins) {
            dbv = nbv - 1 - b / a.nb;
            dbu = a.nb - 1 - (b - (b / a.nb) * a.nb);
            int bv = bv0 - dbv, bu = bu0 - dbu;
            if (bv < 0) bv += a.nby;
            if (bu < 0) bu += a.nbx;
            const int bin = bv * a.nbx + bu;
            beg = __ldg(a.offsets + bin);
            cnt_b = __ldg(a.offsets + bin + 1) - beg;
        }
        int first = cnt_b;   // exclusive scan of the bin sizes
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, first, o);
            if (lane >= o) first += y;
        }
        const int n_cand = __shfl_sync(0xffffffffu, first, 31);
        first -= cnt_b;
        const int nb_here = min(32, nbins - b0);
        for (int c0 = 0; c0 < n_cand; c0 += 32) {
            const int c = c0 + lane;
            // the bin holding candidate c: the last bin whose first index is <= c
            int sel = 0;
            for (int q = 1; q < nb_here; ++q)
                if (__shfl_sync(0xffffffffu, first, q) <= c) sel = q;
            const int my = __shfl_sync(0xffffffffu, beg, sel) + c - __shfl_sync(0xffffffffu, first, sel);
            const int gdbu = __shfl_sync(0xffffffffu, dbu, sel), gdbv = __shfl_sync(0xffffffffu, dbv, sel);
            // the samples of the lane's group that reach this block (bit k: member k)
            unsigned mask = 0u;
            int ru = 0, rvg = 0, p = 0, m_beg = 0;
            unsigned off[8];
            if (c < n_cand) {
                const int2 gd = __ldg(a.gdd + my);
                ru = 4 * gdbu - (gd.x & 3);     // block start relative to the first x tap, >= -3
                rvg = 4 * gdbv - (gd.x >> 2);   // block start relative to the lowest first y cell
                const int cl = gd.y / a.P;
                p = gd.y - cl * a.P;
                m_beg = cstart[cl];
                const int m_cnt = cstart[cl + 1] - m_beg;
                if (ru < a.w && rvg >= -3 && rvg < vspan + a.w) {
                    const int4 o0 = __ldg(a.goff + 2 * my), o1 = __ldg(a.goff + 2 * my + 1);
                    off[0] = o0.x; off[1] = o0.y; off[2] = o0.z; off[3] = o0.w;
                    off[4] = o1.x; off[5] = o1.y; off[6] = o1.z; off[7] = o1.w;
#pragma unroll
                    for (int k = 0; k < kMaxPairsGrouped; ++k) {
                        const int rv = rvg - (int)((off[k >> 1] >> (16 * (k & 1))) & 0xffffu);
                        if (k < m_cnt && rv >= -3 && rv < a.w) mask |= 1u << k;
                    }
                }
            }
            const int cnt = __popc(mask);
            int base = cnt;   // exclusive scan of the counts over the lanes
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, base, o);
                if (lane >= o) base += y;
            }
            const int total = __shfl_sync(0xffffffffu, base, 31);
            base -= cnt;
            if (n + total > kListCap) {   // keep the list within its buffer
                __syncwarp();
                apply(n);
                n = 0;
                __syncwarp();
            }
            int slot = n + base;
            while (mask) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1u;
                // the member's offset: word k / 2, half k % 2 (selected without indexing)
                unsigned word = off[0];
#pragma unroll
                for (int q = 1; q < 8; ++q)
                    if ((k >> 1) == q) word = off[q];
                const int rv = rvg - (int)((word >> (16 * (k & 1))) & 0xffffu);
                const int l = members[m_beg + k] * a.P + p;
                list[slot++] = make_int4(my * nqx + ru + 3, l * rqy + 1 + rv + 3, l, mask == 0u);
            }
            n += total;
        }
    }
    __syncwarp();
    apply(n);
    if constexpr (NF == 2) {
        const int kc = 2 * kg + (lane >> 4);
        if (kc < a.n_kc) {
            float4 *g = reinterpret_cast<float4 *>(a.G + (long long)kc * a.mry * a.mrx * kKC) + (lane & 15);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    g[((long long)(V + j) * a.mrx + (U + i)) * (kKC / 2)] =
                        make_float4(acc[0][j][i].x, acc[0][j][i].y, acc[NF - 1][j][i].x, acc[NF - 1][j][i].y);
        }
    } else {
        float2 *g = a.G + (long long)kg * a.mry * a.mrx * kKC + lane;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) g[((long long)(V + j) * a.mrx + (U + i)) * kKC] = acc[0][j][i];
    }
}

template <int NF, int WARPS, int NS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    spread_groups_kernel(const __grid_constant__ SpreadGroupArgs a) {
    spread_groups_body<NF, WARPS, NS, MINB>(a, blockIdx.x);
}

template <int NF, int WARPS, int NS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    spread_groups_multi(const __grid_constant__ BatchTable<SpreadGroupArgs> t) {
    __shared__ SpreadGroupArgs sa;
    int bid, nb;
    batch_args(t, batch_scan(t, bid, nb), &sa);
    spread_groups_body<NF, WARPS, NS, MINB>(sa, bid);
}

static int spread_groups_describe(const Plan &p, void *ws, SpreadGroupArgs &a) {
    char *w = reinterpret_cast<char *>(ws);
    a.shat = reinterpret_cast<const float2 *>(w + p.off_shat);
    a.gdd = reinterpret_cast<const int2 *>(w + p.off_gdd);
    a.gxq = reinterpret_cast<const float4 *>(w + p.off_gxq);
    a.yq = reinterpret_cast<const float4 *>(w + p.off_yq);
    a.goff = reinterpret_cast<const int4 *>(w + p.off_goff);
    a.offsets = reinterpret_cast<const int *>(w + p.off_offsets);
    a.cls = reinterpret_cast<const int *>(w + p.off_cls);
    a.G = reinterpret_cast<float2 *>(w + p.off_G);
    a.hdr = reinterpret_cast<const WsHeader *>(w);
    a.Lmax = p.L;
    a.P = p.shape.n_pos;
    a.TR = p.shape.n_tx * p.shape.n_rx;
    a.mrx = p.mrx;
    a.mry = p.mry;
    a.nbx = p.nbx;
    a.nby = p.nby;
    a.w = p.w;
    a.nb = (p.w - 1 + kBin - 1) / kBin + 1;
    a.n_kc = p.n_kc;
    const int nf = p.spread_nf, warps = p.spread_warps;
    const int tiles = (p.mrx / (2 * warps)) * (p.mry / 8);
    return tiles * (nf == 2 ? (p.n_kc + 1) / 2 : p.n_kc);
}

template <int NF, int WARPS, int NS, int MINB>
static void spread_groups_launch(const SpreadGroupArgs *a, const BatchTable<SpreadGroupArgs> *t, int blocks,
                                 cudaStream_t s) {
    if (a)
        spread_groups_kernel<NF, WARPS, NS, MINB><<<blocks, WARPS * 32, 0, s>>>(*a);
    else
        spread_groups_multi<NF, WARPS, NS, MINB><<<blocks, WARPS * 32, 0, s>>>(*t);
}

static void spread_groups_dispatch(int key, const SpreadGroupArgs *a, const BatchTable<SpreadGroupArgs> *t,
                                   int blocks, cudaStream_t s) {
    switch (key) {
        case 5: spread_groups_launch<2, 8, 2, 2>(a, t, blocks, s); break;
        case 4: spread_groups_launch<2, 4, 2, 4>(a, t, blocks, s); break;
        case 3: spread_groups_launch<1, 8, 3, 2>(a, t, blocks, s); break;
        default: spread_groups_launch<1, 4, 3, 4>(a, t, blocks, s); break;
    }
}

cudaError_t launch_spread_groups(const Plan &p, void *ws, cudaStream_t s) {
    SpreadGroupArgs a;
    const int blocks = spread_groups_describe(p, ws, a);
    spread_groups_dispatch(2 * p.spread_nf + (p.spread_warps == 8 ? 1 : 0), &a, nullptr, blocks, s);
    return cudaGetLastError();
}

// Both forms: the per-sample scans grouped by launch shape, then the grouped ones.
cudaError_t launch_spread_multi(const mmsar_request *r, int n, cudaStream_t s) {
    std::vector<SpreadArgs> sa((size_t)n);
    std::vector<SpreadGroupArgs> ga((size_t)n);
    std::vector<int> sblocks((size_t)n, 0), gblocks((size_t)n, 0), keys((size_t)n);
    for (int i = 0; i < n; ++i) {
        const Plan &p = r[i].plan->p;
        keys[i] = 2 * p.spread_nf + (p.spread_warps == 8 ? 1 : 0);
        if (p.tc)
            continue;   // tensor-core gridding: launch_grid_tc_multi
        if (p.grouped)
            gblocks[i] = spread_groups_describe(p, r[i].workspace, ga[i]);
        else
            sblocks[i] = spread_describe(p, r[i].workspace, sa[i]);
    }
    cudaError_t e = launch_groups(n, keys.data(), sa.data(), sblocks.data(),
                                  [&](int key, const BatchTable<SpreadArgs> &t, int total) {
                                      spread_dispatch(key, nullptr, &t, total, s);
                                      return cudaGetLastError();
                                  });
    if (e != cudaSuccess) return e;
    return launch_groups(n, keys.data(), ga.data(), gblocks.data(),
                         [&](int key, const BatchTable<SpreadGroupArgs> &t, int total) {
                             spread_groups_dispatch(key, nullptr, &t, total, s);
                             return cudaGetLastError();
                         });
}

}  // namespace mmsar
