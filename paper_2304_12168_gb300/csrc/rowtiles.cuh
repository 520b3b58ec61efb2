// Run-staged row tiles shared by the single-product kernels and the fused chain.
//
// Banded and stencil operands use only a few short runs of x per tile (a 5-point
// stencil: the rows below, at and above the tile). A stage holds one tile's values,
// its 16-bit column slots, its row offsets and only those runs of x: ~21 KB (FP64
// values) or ~12 KB (FP32 values) instead of a whole x window, and HBM moves 10 (6)
// bytes per nonzero instead of 12 (8).
//
// One producer warp fills a ring of stages with 1-D bulk copies; the tile's "full"
// mbarrier expects every byte of the tile at once, so the copies of the matrix part
// (values, slots, row offsets) and of the x runs may be issued at different times:
// the fused chain issues the matrix part of the next product's first tiles before the
// grid-wide barrier that publishes x, and their x runs after it.
#pragma once

#include <cstddef>
#include <cstdint>

#include "internal.h"
#include "mbarrier.cuh"

namespace tacta {

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

template <typename V>
struct __align__(16) TileStageRT {
    static constexpr int kAlign = 16 / (int)sizeof(V);   // values per 16 bytes
    int4 desc;                       // the tile's descriptor (written by the producer)
    V vals[kRunCap + kAlign];
    uint16_t lcol[kRunCap + kPadLcol];
    int32_t rp[kTileRows + 8];
    V xs[kRunXs];
};
using TileStageR = TileStageRT<double>;
using TileStageR32 = TileStageRT<float>;
static_assert(sizeof(TileStageR) % 16 == 0 && sizeof(TileStageR32) % 16 == 0,
              "stage size keeps 16-byte alignment");
static_assert(offsetof(TileStageR, vals) % 16 == 0 && offsetof(TileStageR, lcol) % 16 == 0 &&
              offsetof(TileStageR, rp) % 16 == 0 && offsetof(TileStageR, xs) % 16 == 0,
              "bulk-copy destinations are 16-byte aligned");
static_assert(offsetof(TileStageR32, vals) % 16 == 0 && offsetof(TileStageR32, lcol) % 16 == 0 &&
              offsetof(TileStageR32, rp) % 16 == 0 && offsetof(TileStageR32, xs) % 16 == 0,
              "bulk-copy destinations are 16-byte aligned");

// A tile's descriptor and its kRunMax runs, as the producer warp prefetches them
struct TileMeta {
    int4 d;        // {row begin, row end, nnz begin, nnz end}
    int4 r01, r23; // runs 0..3 as {first, length} pairs
};
static_assert(kRunMax == 4, "TileMeta holds four runs");

__device__ __forceinline__ int4 shfl_int4(const int4 v, int src) {
    return make_int4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// Producer warp: lane i holds the metadata of the block's tile j0 + i, loaded 32 tiles at
// a time, so that lane 0's copy issue never waits on a global load.
struct TilePrefetch {
    TileMeta m{};
    int j0 = -32;
    __device__ __forceinline__ TileMeta get(int j, const int4* __restrict__ tiles, const int2* __restrict__ runs,
                                            int ntiles, int G, int lane) {
        if (j - j0 >= 32) {
            j0 = j;
            const int tl = blockIdx.x + (j0 + lane) * G;
            if (tl < ntiles) {
                m.d = __ldg(tiles + tl);
                const int4* r4 = reinterpret_cast<const int4*>(runs + (size_t)tl * kRunMax);
                m.r01 = __ldg(r4);
                m.r23 = __ldg(r4 + 1);
            }
        }
        const int src = j - j0;
        return TileMeta{shfl_int4(m.d, src), shfl_int4(m.r01, src), shfl_int4(m.r23, src)};
    }
};

// The matrix part of tile tm into stage st (one thread): arms the stage's mbarrier for
// every byte of the tile, x runs included, and copies values, slots and row offsets.
// Copies start on 16-byte boundaries (the padded CSR arrays keep the rounded ends
// inside their allocations).
template <typename V>
__device__ __forceinline__ void tile_issue_mat(const TileMeta& tm, TileStageRT<V>* st, uint64_t* bar,
                                               const int32_t* rowptr, const uint16_t* lcol, const V* vals) {
    constexpr int kA = TileStageRT<V>::kAlign;
    const int4 d = tm.d;
    const int a0 = d.z & ~(kA - 1), c0 = d.z & ~7, r0 = d.x & ~3;
    const uint32_t bv = d.w > d.z ? round16((uint32_t)(d.w - a0) * (uint32_t)sizeof(V)) : 0u;
    const uint32_t bc = d.w > d.z ? round16((uint32_t)(d.w - c0) * 2u) : 0u;
    const uint32_t br = round16((uint32_t)(d.y + 1 - r0) * 4u);
    // run lengths are multiples of 4 entries: 16-byte multiples for both value types
    const uint32_t bx = (uint32_t)(tm.r01.y + tm.r01.w + tm.r23.y + tm.r23.w) * (uint32_t)sizeof(V);
    mbar_expect_tx(bar, bv + bc + br + bx);
    if (bv) bulk_g2s(st->vals, vals + a0, bv, bar);
    if (bc) bulk_g2s(st->lcol, lcol + c0, bc, bar);
    bulk_g2s(st->rp, rowptr + r0, br, bar);
}

// Up to kRunMax runs of x ({first, length} pairs r01, r23) into xs, laid end to end (one thread).
template <typename V>
__device__ __forceinline__ void issue_runs(const int4& r01, const int4& r23, V* xs, uint64_t* bar, const V* x) {
    const int2 rr[kRunMax] = {make_int2(r01.x, r01.y), make_int2(r01.z, r01.w), make_int2(r23.x, r23.y),
                              make_int2(r23.z, r23.w)};
    int off = 0;
#pragma unroll
    for (int k = 0; k < kRunMax; ++k) {
        if (rr[k].y > 0) bulk_g2s(xs + off, x + rr[k].x, (uint32_t)rr[k].y * (uint32_t)sizeof(V), bar);
        off += rr[k].y;
    }
}

// The x runs of tile tm into stage st (one thread; after tile_issue_mat).
template <typename V>
__device__ __forceinline__ void tile_issue_x(const TileMeta& tm, TileStageRT<V>* st, uint64_t* bar, const V* x) {
    issue_runs<V>(tm.r01, tm.r23, st->xs, bar, x);
}

template <typename V>
__device__ __forceinline__ void tile_issue_r(const TileMeta& tm, TileStageRT<V>* st, uint64_t* bar,
                                             const int32_t* rowptr, const uint16_t* lcol, const V* vals,
                                             const V* x) {
    tile_issue_mat<V>(tm, st, bar, rowptr, lcol, vals);
    tile_issue_x<V>(tm, st, bar, x);
}

// One consumer thread's row of a landed tile: warp w of the eight consumer warps owns
// rows [32 w, 32 w + 32) of the tile. Returns the row's dot product (0 for rows past
// the tile's end) and sets row / active.
//   FP64: every lane of the warp runs max(row length) predicated FMA steps, so the warp
//   issues exactly that many FP64 instructions whatever the spread of lengths.
//   FP32: a plain loop over the row.
__device__ __forceinline__ double rw_row_dot(const TileStageR* Sg, int warp, int lane, int& row, bool& active) {
    const int4 d = Sg->desc;
    row = d.x + warp * 32 + lane;
    active = row < d.y;
    int kb = 0, len = 0;
    if (active) {
        const int r0 = d.x & ~3;
        kb = Sg->rp[row - r0];
        len = Sg->rp[row + 1 - r0] - kb;
    }
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    const int vb = kb - (d.z & ~1), cb = kb - (d.z & ~7);
    double sum = 0.0;
    for (int u = 0; u < maxlen; ++u)
        if (u < len) sum = fma(Sg->vals[vb + u], Sg->xs[Sg->lcol[cb + u]], sum);
    return sum;
}

__device__ __forceinline__ float rw_row_dot(const TileStageR32* Sg, int warp, int lane, int& row, bool& active) {
    const int4 d = Sg->desc;
    row = d.x + warp * 32 + lane;
    active = row < d.y;
    int kb = 0, len = 0;
    if (active) {
        const int r0 = d.x & ~3;
        kb = Sg->rp[row - r0];
        len = Sg->rp[row + 1 - r0] - kb;
    }
    const int vb = kb - (d.z & ~3), cb = kb - (d.z & ~7);
    float sum = 0.0f;
    for (int u = 0; u < len; ++u) sum = fmaf(Sg->vals[vb + u], Sg->xs[Sg->lcol[cb + u]], sum);
    return sum;
}

// ------------------------------------------------------------------ tile formats
//
// A format supplies the stage layout, the per-tile metadata the producer warp prefetches,
// the copy issue (matrix part, then x runs) and the row dot product of one consumer lane.

// Run-staged CSR: values, 16-bit column slots and row offsets per tile (any banded CSR
// whose tiles draw on at most four short runs of x).
template <typename V>
struct RunFmt {
    using Stage = TileStageRT<V>;
    using Meta = TileMeta;
    using Ops = ChainOps<V>;
    struct Prefetch {
        TilePrefetch pf;
        __device__ __forceinline__ Meta get(int j, const Ops& ops, int o, int G, int lane) {
            return pf.get(j, ops.tiles[o], ops.runs[o], ops.ntiles[o], G, lane);
        }
    };
    static __device__ __forceinline__ void issue_mat(const Meta& m, Stage* st, uint64_t* bar, const Ops& ops, int o) {
        st->desc = m.d;   // visible to the consumers through the stage's mbarrier
        tile_issue_mat<V>(m, st, bar, ops.rowptr[o], ops.lcol[o], ops.vals[o]);
    }
    static __device__ __forceinline__ void issue_x(const Meta& m, Stage* st, uint64_t* bar, const V* x) {
        tile_issue_x<V>(m, st, bar, x);
    }
    static __device__ __forceinline__ V row_dot(const Stage* sg, const Ops&, int warp, int lane, int& row,
                                                bool& active) {
        return rw_row_dot(sg, warp, lane, row, active);
    }
};

// Diagonal form (DIA): every nonzero on one of k <= kDiaMax diagonals col - row = offset_k.
// A tile's stage holds its k x 256 values laid out by diagonal then row, one byte per
// row with bit k set where the row stores diagonal k, and its runs of x; lane r of the
// tile reads x[row0 + r + offset_k] at slot sbase_k + r. Per nonzero only its value moves
// (8 bytes FP64, 4 FP32), against 10 / 6 with the run-staged CSR's slots and offsets, and
// the row's FMAs run in ascending diagonal order, i.e. ascending column: that is the CSR
// order, and the products equal the CSR kernels' bit for bit, when each CSR row lists its
// columns in ascending order (the transposes built here always do; a caller's A with
// unsorted rows can differ in the last bits).
template <typename V>
struct __align__(16) DiaStage {
    int4 desc;                       // {row begin, row end, tile, 0}
    int32_t sbase[8];                // slot of x[row begin + offset_k] in xs
    uint8_t mask[kTileRows];
    V vals[kDiaMax * kTileRows];
    V xs[kRunXs];
};
static_assert(offsetof(DiaStage<double>, mask) % 16 == 0 && offsetof(DiaStage<double>, vals) % 16 == 0 &&
              offsetof(DiaStage<double>, xs) % 16 == 0 && sizeof(DiaStage<double>) % 16 == 0 &&
              offsetof(DiaStage<float>, vals) % 16 == 0 && offsetof(DiaStage<float>, xs) % 16 == 0 &&
              sizeof(DiaStage<float>) % 16 == 0, "bulk-copy destinations are 16-byte aligned");
static_assert(kDiaMax <= 8, "DiaStage holds eight slot bases");

struct DiaMeta {
    int4 d;          // {row begin, row end, tile, 0}
    int4 r01, r23;   // runs 0..3 as {first, length} pairs
    int4 s0, s1;     // slot bases of diagonals 0..7
};

template <typename V>
struct DiaFmt {
    using Stage = DiaStage<V>;
    using Meta = DiaMeta;
    using Ops = ChainOpsDia<V>;
    struct Prefetch {   // lane i holds tile j0 + i's runs and slot bases, 32 tiles at a time
        int4 r01{}, r23{}, s0{}, s1{};
        int j0 = -32;
        __device__ __forceinline__ Meta get(int j, const Ops& ops, int o, int G, int lane) {
            if (j - j0 >= 32) {
                j0 = j;
                const int tl = blockIdx.x + (j0 + lane) * G;
                if (tl < ops.ntiles[o]) {
                    const int4* r4 = reinterpret_cast<const int4*>(ops.runs[o] + (size_t)tl * kRunMax);
                    r01 = __ldg(r4);
                    r23 = __ldg(r4 + 1);
                    const int4* s4 = reinterpret_cast<const int4*>(ops.sbase[o] + (size_t)tl * 8);
                    s0 = __ldg(s4);
                    s1 = __ldg(s4 + 1);
                }
            }
            const int src = j - j0;
            const int tl = blockIdx.x + j * G;
            const int r0 = tl * kTileRows;
            const int r1 = r0 + kTileRows < ops.rows[o] ? r0 + kTileRows : ops.rows[o];
            return Meta{make_int4(r0, r1, tl, 0), shfl_int4(r01, src), shfl_int4(r23, src), shfl_int4(s0, src),
                        shfl_int4(s1, src)};
        }
    };
    static __device__ __forceinline__ void issue_mat(const Meta& m, Stage* st, uint64_t* bar, const Ops& ops, int o) {
        st->desc = m.d;
        st->sbase[0] = m.s0.x; st->sbase[1] = m.s0.y; st->sbase[2] = m.s0.z; st->sbase[3] = m.s0.w;
        st->sbase[4] = m.s1.x; st->sbase[5] = m.s1.y; st->sbase[6] = m.s1.z; st->sbase[7] = m.s1.w;
        const uint32_t bv = (uint32_t)ops.k * kTileRows * (uint32_t)sizeof(V);
        const uint32_t bx = (uint32_t)(m.r01.y + m.r01.w + m.r23.y + m.r23.w) * (uint32_t)sizeof(V);
        mbar_expect_tx(bar, bv + kTileRows + bx);
        bulk_g2s(st->vals, ops.vals[o] + (size_t)m.d.z * ops.k * kTileRows, bv, bar);
        bulk_g2s(st->mask, ops.mask[o] + (size_t)m.d.z * kTileRows, kTileRows, bar);
    }
    static __device__ __forceinline__ void issue_x(const Meta& m, Stage* st, uint64_t* bar, const V* x) {
        issue_runs<V>(m.r01, m.r23, st->xs, bar, x);
    }
    static __device__ __forceinline__ V row_dot(const Stage* sg, const Ops& ops, int warp, int lane, int& row,
                                                bool& active) {
        const int lr = warp * 32 + lane;
        row = sg->desc.x + lr;
        active = row < sg->desc.y;
        const unsigned msk = active ? sg->mask[lr] : 0u;
        V sum = V(0);
#pragma unroll
        for (int k = 0; k < kDiaMax; ++k)
            if (k < ops.k && ((msk >> k) & 1u)) sum = fma(sg->vals[k * kTileRows + lr], sg->xs[sg->sbase[k] + lr], sum);
        return sum;
    }
};

// eight consumer warps (one per 32 rows of a tile) and one producer warp
constexpr int kRwConsumers = kTileRows / 32;
constexpr int kRwThreads = (kRwConsumers + 1) * 32;
constexpr int kRw32Stages = 4, kRw32BlocksPerSM = 4;

}  // namespace tacta
