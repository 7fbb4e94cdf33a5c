"""Tile orders of the tensor-core GEMM's persistent loop (fmx_tile_order, CPU only).

A launch of G CTAs walks positions t = i, i + G, ... per CTA i, and the decode of t picks a
tile.  A wrong decode would skip or repeat tiles without any fault (the product would just be
wrong where the parity tests happen not to look), so the decode is checked here against its
definition for many shapes and grids: every order is a bijection onto the launch's tiles (the
Hermitian order onto the tiles on or above the diagonal only).  The balance the paired orders
exist for is checked with the K-block counts of the triangular products (row block r of a
lower-triangular A spans r + 1 diagonal blocks, of an upper one mt_mod - r; column tile c of an
upper-triangular B spans c + 1): at the Cholesky recursion's large sizes no CTA carries more
than 6 % above the mean (13-18 % at the smaller or one-item launches), where the plain raster
left the triangular-A products up to 1.24x (152 CTAs) and 1.53x (144).
"""
import ctypes

import numpy as np
import pytest

RASTER, PAIRS_A, PAIRS_B, HERM = 0, 1, 2, 3


@pytest.fixture(scope="module")
def order():
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm
    f = fm.lib.fmx_tile_order
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 6 + [ctypes.c_void_p, ctypes.c_int]

    def run(kind, mt_mod, ntn, batch, lower, grid):
        cap = batch * 2 * mt_mod * ntn
        out = np.full(3 * cap, -1, dtype=np.int32)
        n = f(kind, mt_mod, ntn, batch, lower, grid, out.ctypes.data, cap)
        assert n >= 0, (kind, mt_mod, ntn, batch, grid)
        return out[:3 * n].reshape(n, 3), min(grid, n)
    return run


def expected(kind, mt_mod, ntn, batch):
    return {(mt, nt, b) for b in range(batch) for mt in range(2 * mt_mod) for nt in range(ntn)
            if kind != HERM or mt % mt_mod <= nt}


def kwork(kind, lower, mt_mod, mt, nt):
    r = mt % mt_mod
    if kind == PAIRS_A:
        return r + 1 if lower else mt_mod - r
    if kind == PAIRS_B:
        return nt + 1
    return 1


SHAPES = [(1, 1), (2, 2), (4, 4), (8, 8), (16, 16), (32, 32), (4, 6), (10, 2), (64, 64)]


@pytest.mark.parametrize("kind", [RASTER, PAIRS_A, PAIRS_B, HERM])
def test_every_order_is_a_bijection_onto_its_tiles(order, kind):
    for mt_mod, ntn in SHAPES:
        if (kind == PAIRS_A and mt_mod % 2) or (kind == PAIRS_B and ntn % 2) or (kind == HERM and ntn != mt_mod):
            continue
        for batch in (1, 2, 3):
            for grid in (1, 7, 144, 152, 100000):
                for lower in ((0, 1) if kind == PAIRS_A else (0,)):
                    tiles, _ = order(kind, mt_mod, ntn, batch, lower, grid)
                    got = [tuple(t) for t in tiles]
                    assert len(got) == len(set(got)), (kind, mt_mod, ntn, batch, grid)
                    assert set(got) == expected(kind, mt_mod, ntn, batch), (kind, mt_mod, ntn, batch, grid)


def test_invalid_arguments_are_refused(order):
    from paper_2508_18468_gb300 import fm
    f = fm.lib.fmx_tile_order
    buf = np.zeros(3 * 64, dtype=np.int32)
    assert f(PAIRS_A, 3, 4, 1, 1, 8, buf.ctypes.data, 64) == -1      # odd row-block count
    assert f(PAIRS_B, 4, 3, 1, 0, 8, buf.ctypes.data, 64) == -1      # odd column-tile count
    assert f(HERM, 4, 5, 1, 0, 8, buf.ctypes.data, 64) == -1         # not square
    assert f(7, 4, 4, 1, 0, 8, buf.ctypes.data, 64) == -1            # unknown order
    assert f(RASTER, 4, 4, 2, 0, 8, buf.ctypes.data, 63) == -1       # 64 tiles do not fit
    assert f(RASTER, 4, 4, 1, 0, 8, None, 64) == -1                  # no output array


def _imbalance(tiles, G, kind, lower, mt_mod):
    load = np.zeros(G)
    for t, (mt, nt, b) in enumerate(tiles):
        load[t % G] += kwork(kind, lower, mt_mod, mt, nt)
    return load.max() / load.mean()


@pytest.mark.parametrize("grid", [144, 152])
def test_paired_orders_balance_the_triangular_products(order, grid):
    # the Cholesky recursion's largest products: blocks of 4096 (32 row tiles) and 2048 (16),
    # two trajectories per half of the batch, or one per chain; 144 CTAs when the halves run
    # side by side (8 SMs left to the other half), 152 otherwise.  What is left above 1 is the
    # last, partial round (whole tiles cannot split it evenly).
    for mt_mod, batch, bound in ((32, 2, 1.06), (32, 1, 1.13), (16, 2, 1.18)):
        for kind, lower in ((PAIRS_A, 1), (PAIRS_A, 0), (PAIRS_B, 0)):
            tiles, G = order(kind, mt_mod, mt_mod, batch, lower, grid)
            paired = _imbalance(tiles, G, kind, lower, mt_mod)
            rtiles, _ = order(RASTER, mt_mod, mt_mod, batch, 0, grid)
            raster = _imbalance(rtiles, G, kind, lower, mt_mod)
            assert paired <= bound, (kind, lower, mt_mod, batch, grid, paired)
            if kind == PAIRS_A:
                # the raster leaves 1.24x (152 CTAs) to 2.1x (144, 16 row tiles) here
                assert paired < raster - 0.15, (kind, lower, mt_mod, batch, grid, paired, raster)
            else:
                # triangular B: the raster's sweep along the columns already mixes the K ranges
                # (1.03-1.24x); the pairing stays within 3 % of it and is better where it is worst
                assert paired <= 1.03 * raster, (kind, lower, mt_mod, batch, grid, paired, raster)


def test_hermitian_order_gives_every_cta_the_same_count_within_one(order):
    for mt_mod, batch in ((32, 2), (32, 1), (16, 2), (8, 3)):
        tiles, G = order(HERM, mt_mod, mt_mod, batch, 0, 152)
        counts = np.bincount(np.arange(len(tiles)) % G, minlength=G)
        assert counts.max() - counts.min() <= 1
        # rows within a column first, in groups of 16 row tiles: the first 16 positions of
        # a (batch item, half) are column 0's row 0, column 1's rows 0-1, ...
        assert [tuple(t) for t in tiles[:3]] == [(0, 0, 0), (0, 1, 0), (1, 1, 0)]
