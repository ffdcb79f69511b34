"""Pins of the oracle's cell keys and stable sort: keys against an independent computation
from absolute positions (floor(x/dx - 1/2) / floor(x/dx) - 1 stencil base of Sec. 3.5 on a
power-of-two spacing, where the division is exact), and the sort against numpy's stable
argsort."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("edge", [4, 8])
def test_keys_match_floor_rule(dim, order, edge):
    res = 64
    dx = 1.0 / 64
    cfg = oracle.make_cfg(dim=dim, order=order, res=(res,) * dim, dx=dx)
    rng = np.random.default_rng(0)
    n = 5000
    cell = rng.integers(4, res - 5, size=(n, dim)).astype(np.int32)
    off = rng.random((n, dim))
    off[:50] = 0.5          # ties sit exactly on the quadratic switch point
    off[50:100] = 0.0
    got = oracle.keys(cfg, edge, cell, off)
    x = (cell + off) * dx
    u = x / dx
    base = np.floor(u - 0.5).astype(np.int64) if order == 2 else np.floor(u).astype(np.int64) - 1
    nb = (res + edge - 1) // edge
    lg = int(np.log2(edge))
    blk = np.zeros(n, dtype=np.int64)
    inn = np.zeros(n, dtype=np.int64)
    for a in reversed(range(dim)):
        blk = blk * nb + base[:, a] // edge
        inn = inn * edge + base[:, a] % edge
    exp = (blk << (dim * lg)) | inn
    np.testing.assert_array_equal(got.astype(np.int64), exp)


def test_stable_sort_matches_numpy():
    rng = np.random.default_rng(1)
    for n in (0, 1, 7, 1000, 100_000):
        k = rng.integers(0, 50, size=n).astype(np.uint32)
        np.testing.assert_array_equal(oracle.stable_sort(k), np.argsort(k, kind="stable"))
