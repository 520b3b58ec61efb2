// Per-tile plan of the diagonal form, compiled for the device (the plan-time kernel) and
// for the host (exported as tacta_dia_tile_plan, so the index arithmetic is checked on the
// CPU against a brute-force construction).
//
// For a tile of kTileRows rows starting at r0 and k diagonals col - row = off[i]
// (ascending), diagonal i touches x[r0 + off[i] .. r1 + off[i]) clipped to [0, cols).
// Each range is aligned outwards to 4 entries (16-byte bulk copies in FP32 and FP64),
// ranges closer than kRunGap are merged into one run, and the runs are laid end to end
// in the stage; row r of the tile finds x[r + off[i]] at slot sbase[i] + (r - r0).
// The tile fits when it needs at most kRunMax runs of at most kRunXs entries in total.
#pragma once

#include <cstdint>

#include "internal.h"

namespace tacta {

struct DiaOffsets {
    int k;
    int off[kDiaMax];
};

// runs: kRunMax {first, length} pairs (unused: {0, 0}); sbase: 8 slot bases (unused: 0).
// Returns whether the tile fits; runs and sbase are written only when it does.
__host__ __device__ inline bool dia_tile_plan(int64_t rows, int64_t cols, const DiaOffsets& d, int t, int2* runs,
                                              int32_t* sbase) {
    const int64_t r0 = (int64_t)t * kTileRows;
    const int64_t r1 = r0 + kTileRows < rows ? r0 + kTileRows : rows;
    int2 rr[kRunMax];
    int rk[kDiaMax];
    int nrun = 0, total = 0;
    bool bad = false;
    int64_t cs = -1, ce = -1;   // the run being merged, [cs, ce)
    for (int k = 0; k < d.k; ++k) {
        rk[k] = -1;
        int64_t s = r0 + d.off[k], e = r1 + d.off[k];
        if (s < 0) s = 0;
        if (e > cols) e = cols;
        if (s >= e) continue;
        s &= ~(int64_t)3;
        e = (e + 3) & ~(int64_t)3;
        if (cs >= 0 && s <= ce + kRunGap) {
            if (e > ce) ce = e;
        } else {
            if (cs >= 0) {
                if (nrun == kRunMax) { bad = true; break; }
                rr[nrun++] = make_int2((int)cs, (int)(ce - cs));
                total += (int)(ce - cs);
            }
            cs = s;
            ce = e;
        }
        rk[k] = nrun;   // the index the run being merged gets when it closes
    }
    if (!bad && cs >= 0) {
        if (nrun == kRunMax) {
            bad = true;
        } else {
            rr[nrun++] = make_int2((int)cs, (int)(ce - cs));
            total += (int)(ce - cs);
        }
    }
    if (bad || total > kRunXs) return false;
    int start[kRunMax];
    for (int i = 0, o = 0; i < kRunMax; ++i) {
        start[i] = o;
        if (i < nrun) o += rr[i].y;
    }
    for (int i = 0; i < kRunMax; ++i) runs[i] = i < nrun ? rr[i] : make_int2(0, 0);
    for (int k = 0; k < 8; ++k) {
        int sb = 0;
        if (k < d.k && rk[k] >= 0) sb = start[rk[k]] + (int)(r0 + d.off[k] - rr[rk[k]].x);
        sbase[k] = sb;
    }
    return true;
}

}  // namespace tacta
