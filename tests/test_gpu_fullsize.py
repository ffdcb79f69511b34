"""Parity at the benchmark's full size and launch configuration (128^3 grid, elastic cube of
side 0.4 at 32 particles per cell = 4.29M particles, FP32, quadratic, fixed-corotated,
gravity, sticky walls, default tile and P2G kernel, as bench.py runs it):

- cell keys and the stable sort permutation, every particle, bit-exact;
- P2G at every grid node, against the oracle's P2G of all particles;
- the grid update on the whole grid;
- G2P on every particle, from the GPU's grid velocities;
- the next step's sort (keys written by G2P, sorted incrementally), bit-exact against the
  stable sort of keys recomputed from the new positions
  (a particle that G2P skipped or wrote twice shows up here).
The initial state is deformed and moving (random F, v, B) so every term is exercised."""
import numpy as np
import pytest

import oracle
from helpers import kappa, nodewise_err, particlewise_err, relerr, stencil_max_speed
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_1603_06188_gb300 import apic

    apic.load(build_if_missing=True)
    w = dict(bench.WORKLOADS["cube128"])
    sc = scenes.falling_cube_3d(res=128, side=0.4, ppc=32, seed=7, omega=(0.3, -0.5, 1.0), v0=(0.2, 0.0, -0.1))
    rng = np.random.default_rng(7)
    x = sc.x
    v = sc.v + 0.05 * rng.normal(size=sc.v.shape)
    B = sc.grad_v * kappa(2) * sc.dx ** 2 + 1e-6 * rng.normal(size=(sc.n, 3, 3))
    F = scenes.random_deformation(rng, sc.n, 3, 0.05)
    cfg = bench.lib_config(w, sc)
    sim = apic.Sim(cfg, sc.n)
    sim.upload(x, v, B, F)
    x0, v0, B0, F0 = sim.download()
    cell0, off0 = sim.download_positions()
    sim.p2g()
    keys, perm = sim.keys()
    m_g, p_g = sim.grid("momentum")
    sim.grid_update()
    m_v, vt = sim.grid("velocity")
    sim.g2p()
    out = sim.download()
    cell1, off1 = sim.download_positions()
    sim.p2g()                                   # sorts the keys written by G2P
    keys1, perm1 = sim.keys()
    sim.close()
    oc = bench.oracle_config(w, sc)
    vol = sc.dx ** 3 / w["ppc"]
    return dict(sc=sc, oc=oc, vol=vol, mass=w["rho"] * vol, x0=x0, v0=v0, B0=B0, F0=F0, cell0=cell0, off0=off0,
                keys=keys, perm=perm, m_g=m_g, p_g=p_g, m_v=m_v, vt=vt, out=out, cell1=cell1, off1=off1, keys1=keys1, perm1=perm1)


def test_fullsize_keys_and_sort_bit_exact(run):
    ref_keys = oracle.keys(run["oc"], 4, run["cell0"], run["off0"])
    ref_perm = oracle.stable_sort(ref_keys)
    np.testing.assert_array_equal(run["keys"], ref_keys[ref_perm])
    np.testing.assert_array_equal(run["perm"].astype(np.int64), ref_perm)


def test_fullsize_p2g_every_node(run):
    """The oracle's P2G over all 4.29M particles (about 15 s on one core) against the GPU's
    grid at every node of the 128^3 grid: mass and momentum normwise, and the set of nodes
    that hold mass."""
    oc = run["oc"]
    gm, gmv, gf, bad = oracle.p2g(oc, run["x0"], run["v0"], run["B0"], run["F0"], run["mass"], run["vol"])
    assert bad == 0
    ref_p = gmv + oc.dt * gf
    assert relerr(run["m_g"], gm) <= TOL
    assert relerr(run["p_g"], ref_p) <= TOL
    np.testing.assert_array_equal(run["m_g"] > 0, gm > 0)
    # every node, against its own scale (a node with little mass gets a tighter bound than
    # the normwise one), so an error confined to a few tiles cannot hide
    assert nodewise_err(run["m_g"], gm, gm) <= TOL
    assert nodewise_err(run["p_g"], ref_p, gm) <= TOL


def test_fullsize_grid_update(run):
    oc = run["oc"]
    _, vt_ref = oracle.grid_update(oc, run["m_g"], run["p_g"], np.zeros_like(run["p_g"]))
    np.testing.assert_array_equal(run["m_v"], run["m_g"])
    assert relerr(run["vt"], vt_ref) <= TOL


def test_fullsize_g2p_every_particle(run):
    oc = run["oc"]
    idx = np.arange(run["sc"].n)
    x1, v1, B1, F1, bad = oracle.g2p(oc, run["x0"], run["F0"], run["vt"], run["vt"])
    assert bad == 0
    gx, gv, gB, gF = (a[idx] for a in run["out"])
    assert relerr(gv, v1) <= TOL
    assert relerr(gB, B1) <= TOL
    assert relerr(gF, F1) <= TOL
    smax = stencil_max_speed(run["x0"], run["vt"], (128,) * 3, oc.dx, 2)
    assert particlewise_err(gv, v1, smax) <= TOL
    assert particlewise_err(gB, B1, smax * oc.dx) <= TOL
    # positions are cell + FP32 offset: one rounding of the offset is eps32 * dx absolute,
    # which at dt = 2e-5 is not small against the displacement itself
    disp_ref = x1 - run["x0"][idx]
    bound = TOL * np.abs(disp_ref).max() + 2 * np.finfo(np.float32).eps * run["sc"].dx
    assert np.abs((gx - run["x0"][idx]) - disp_ref).max() <= bound


def test_fullsize_next_sort_bit_exact(run):
    # after G2P the particles are stored in the first step's sorted order, so the keys G2P
    # wrote are, in storage order, the oracle's keys of particle perm[k] at k
    by_id = oracle.keys(run["oc"], 4, run["cell1"], run["off1"])
    knext = by_id[run["perm"].astype(np.int64)]
    ref_perm = oracle.stable_sort(knext)
    np.testing.assert_array_equal(run["keys1"], knext[ref_perm])
    np.testing.assert_array_equal(run["perm1"].astype(np.int64), ref_perm)
