"""The stable sort of cell keys after a step, when only the particles whose key changed are
sorted and merged into the already-sorted rest (the particles are then stored in the previous
sorted order).  Each step's keys and permutation are compared bit for bit with the oracle's
stable sort of the keys recomputed from the downloaded positions, for a few moved particles
(less than one radix tile), for many (several tiles), and for every particle moving."""
import numpy as np
import pytest

import oracle
from helpers import configs
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic as mod

    mod.load(build_if_missing=True)
    return mod


def run_and_check(apic, res, side, ppc, vel, steps, dt=2e-5, min_moved=0, tile=0):
    sc = scenes.falling_cube_3d(res=res, side=side, ppc=ppc, seed=3)
    v = vel(np.random.default_rng(4), sc.n)
    gc, oc, m, vol = configs(3, 2, (res,) * 3, sc.dx, dt=dt, gravity=(0.0, 0.0, 0.0), boundary="none", wall=3,
                             vol=sc.dx ** 3 / ppc, mass=sc.dx ** 3 / ppc, tile=tile, model="none")
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, v, np.zeros((sc.n, 3, 3)), np.broadcast_to(np.eye(3), (sc.n, 3, 3)))
    ids = np.arange(sc.n)          # particle id stored at each index
    prev = None
    moved_seen = []
    for step in range(steps):
        cell, off = sim.download_positions()
        by_id = oracle.keys(oc, 4, cell, off)
        knext = by_id[ids]          # keys in storage order
        sim.p2g()
        keys, perm = sim.keys()
        ref_perm = oracle.stable_sort(knext)
        np.testing.assert_array_equal(keys, knext[ref_perm], err_msg=f"step {step}")
        np.testing.assert_array_equal(perm.astype(np.int64), ref_perm, err_msg=f"step {step}")
        if prev is not None:
            moved_seen.append(int(np.count_nonzero(knext != prev)))
        sim.grid_update()
        sim.g2p()
        ids = ids[perm.astype(np.int64)]
        prev = keys.astype(np.uint32)
    sim.download()
    sim.close()
    assert min(moved_seen) >= min_moved, moved_seen
    return moved_seen


def test_resort_few_moved(apic):
    # slow, smooth motion: a handful of particles change cell per step (m < one radix tile)
    moved = run_and_check(apic, 32, 0.5, 8, lambda rng, n: np.tile([0.8, -0.5, 0.3], (n, 1)), steps=5)
    assert max(moved) < 2048


def test_resort_many_moved(apic):
    # fast rigid rotation: a large fraction moves each step (m spans several radix tiles)
    res = 64
    sc = scenes.falling_cube_3d(res=res, side=0.5, ppc=8, seed=3)
    w = np.array([120.0, -80.0, 200.0])
    v_of = lambda rng, n: np.cross(w, sc.x - 0.5)
    run_and_check(apic, res, 0.5, 8, v_of, steps=4, min_moved=4096)


def test_resort_all_moved(apic):
    # a uniform displacement of one cell per step changes every particle's base cell
    dt, res = 2e-5, 32
    speed = 1.0 / res / dt
    moved = run_and_check(apic, res, 0.3, 8, lambda rng, n: np.tile([speed, 0.0, 0.0], (n, 1)), steps=3, dt=dt)
    n_particles = len(scenes.falling_cube_3d(res=res, side=0.3, ppc=8, seed=3).x)
    assert min(moved) > 0.9 * n_particles


def test_resort_small_tiles(apic):
    # tile list built from the merged order at the smallest tile size
    sc = scenes.falling_cube_3d(res=32, side=0.5, ppc=8, seed=3)
    w = np.array([0.0, 150.0, -100.0])
    run_and_check(apic, 32, 0.5, 8, lambda rng, n: np.cross(w, sc.x - 0.5), steps=3, tile=256)


def test_resort_collapse(apic):
    # an affine velocity field that carries every particle 90 % of the way to the centre in
    # one step: the changed keys crowd into a few node blocks, so a chunk of the previous
    # order owns far more changed keys than the merge stages in shared memory
    dt, res = 2e-5, 32
    sc = scenes.falling_cube_3d(res=res, side=0.5, ppc=8, seed=3)
    centre = sc.x.mean(axis=0)
    moved = run_and_check(apic, res, 0.5, 8, lambda rng, n: -(sc.x - centre) * (0.9 / dt), steps=3, dt=dt)
    assert moved[0] > 0.9 * sc.n
