"""The per-tile plan of the diagonal form (tacta_dia_tile_plan: the code the plan-time
kernel runs, compiled for the host), checked on the CPU against a brute-force
construction: every entry a row of the tile can store is found at its slot, the staged
runs are aligned and inside the padded vector, and a tile is accepted exactly when the
merged runs respect the stage's limits (4 runs, 896 entries)."""
import numpy as np
import pytest

import paper_2304_12168_gb300 as tacta

TILE, RUN_MAX, RUN_XS, GAP = 256, 4, 896, 16


@pytest.fixture(scope="module")
def lib():
    return tacta.load_library()


def brute_runs(rows, cols, offsets, tile):
    """Each diagonal's column range over the tile's rows, clipped and aligned outwards to 4,
    merged when the gap is at most 16: the runs the stage must hold."""
    r0, r1 = tile * TILE, min(tile * TILE + TILE, rows)
    ranges = []
    for o in offsets:
        s, e = max(r0 + o, 0), min(r1 + o, cols)
        if s < e:
            ranges.append((s & ~3, (e + 3) & ~3))
    runs = []
    for s, e in sorted(ranges):
        if runs and s <= runs[-1][1] + GAP:
            runs[-1][1] = max(runs[-1][1], e)
        else:
            runs.append([s, e])
    return [(s, e - s) for s, e in runs]


def check(rows, cols, offsets, tile):
    fits, runs, sb = tacta.dia_tile_plan(rows, cols, offsets, tile)
    want = brute_runs(rows, cols, offsets, tile)
    want_fits = len(want) <= RUN_MAX and sum(l for _, l in want) <= RUN_XS
    assert fits == want_fits, (rows, cols, offsets, tile, want)
    if not fits:
        return False
    used = [r for r in runs if r[1] > 0]
    assert used == want
    assert all(r == (0, 0) for r in runs[len(used):])
    staged = np.concatenate([np.arange(f, f + l) for f, l in used]) if used else np.zeros(0, int)
    for f, l in used:
        assert f % 4 == 0 and l % 4 == 0 and l > 0 and f >= 0 and f + l <= ((cols + 3) & ~3)
    r0, r1 = tile * TILE, min(tile * TILE + TILE, rows)
    for k, o in enumerate(offsets):
        for r in range(r0, r1):
            c = r + o
            if 0 <= c < cols:
                slot = sb[k] + (r - r0)
                assert 0 <= slot < len(staged) and staged[slot] == c, (offsets, tile, r, k)
    assert all(v == 0 for v in sb[len(offsets):])
    return True


@pytest.mark.parametrize("width", [24, 300, 1000, 3000])
def test_stencil_tiles(lib, width):
    """2D 5-point stencils: every tile fits (three runs, or one when the grid is narrow)."""
    n = width * width
    offs = [-width, -1, 0, 1, width]
    ntiles = -(-n // TILE)
    for t in sorted({0, 1, 2, ntiles // 2, ntiles - 2, ntiles - 1}):
        assert check(n, n, offs, t)


def test_rectangular_and_ragged_last_tile(lib):
    """20000 x 22000 with diagonals 0, 700, 1500 (A) and its transpose's -1500, -700, 0; the
    last tile holds 32 rows."""
    for t in (0, 1, 40, 77, 78):
        assert check(20000, 22000, [0, 700, 1500], t)
    for t in (0, 5, 84, 85):
        assert check(22000, 20000, [-1500, -700, 0], t)


def test_tridiagonal_and_far_diagonals(lib):
    for t in (0, 100, 390):
        assert check(100001, 100001, [-1, 1], t)
    # diagonals entirely outside the matrix for some tiles: those ranges are empty
    for t in (0, 3, 7):
        assert check(2000, 2000, [-1800, 0, 1800], t)


def test_tiles_that_do_not_fit(lib):
    """Five separated ranges (a 3D 7-point pattern has more): more runs than a stage holds;
    a band 1000 wide: one run of more than 896 entries."""
    assert not check(10 ** 6, 10 ** 6, [-10000, -100, 0, 100, 10000], 100)
    assert not check(10 ** 5, 10 ** 5, [-500, -250, 0, 250, 500], 50)


def test_random_offset_sets(lib):
    rng = np.random.default_rng(21)
    accepted = 0
    for _ in range(150):
        rows = int(rng.integers(1, 5000))
        cols = int(rng.integers(1, 5000))
        k = int(rng.integers(1, 6))
        offs = sorted(set(int(v) for v in rng.integers(-1200, 1200, size=k)))
        tile = int(rng.integers(0, -(-rows // TILE)))
        accepted += check(rows, cols, offs, tile)
    assert 0 < accepted < 150      # both outcomes exercised


def test_invalid_arguments(lib):
    assert tacta.dia_tile_plan(100, 100, [0, 1], 1)[0] is None          # tile past the last row
    assert tacta.dia_tile_plan(100, 100, [1, 0], 0)[0] is None          # offsets not ascending
    assert tacta.dia_tile_plan(100, 100, [0, 1, 2, 3, 4, 5], 0)[0] is None   # more than five
    assert tacta.dia_tile_plan(0, 100, [0], 0)[0] is None
