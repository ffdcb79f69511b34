"""Batched stepping: many simulations of different sizes, grids and materials advanced
together must give, for each member, the state that stepping it alone gives (to FP32
rounding: the order of the floating-point additions into shared grid nodes differs), with
and without CUDA-graph capture, through membership changes and the autotuner."""
import numpy as np
import pytest

from helpers import kappa, relerr
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


def make_members(apic, count, seed=0, dim=3, order=2, precision=32, ppc=8):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        spec = scenes.random_sim_spec(rng, edge_range=(24, 40), np_range=(2000, 30000))
        if dim == 3:
            sc = scenes.sim_from_spec(spec, ppc=ppc)
        else:
            sc = scenes.rotating_disk_2d(res=spec["edge"] * 2, radius=0.2, ppc=4, seed=spec["seed"], omega=1.0)
        k = kappa(order) * sc.dx ** 2
        B = sc.grad_v * k
        F = scenes.random_deformation(rng, sc.n, dim, 0.05)
        E = float(rng.uniform(5e3, 5e4))
        vol = sc.dx ** dim / ppc
        cfg = apic.make_config(dim=dim, order=order, precision=precision, res=sc.res, dx=sc.dx, dt=2e-5,
                               gravity=(0.0, -9.8, 0.0)[:dim] if i % 2 else (0.0,) * dim, boundary="sticky",
                               wall=order + 1, model="fcr", E=E, nu=0.3, particle_mass=vol, particle_volume=vol)
        out.append((cfg, sc.x, sc.v, B, F))
    return out


def run_alone(apic, members, steps):
    res = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        sim.step(steps)
        res.append(sim.download())
        sim.close()
    return res


# Under rigid motion B_p = sum_i w v_i (x_i - x_p)^T is a small difference of terms about
# |x_p - axis| / dx times larger, so the rounding of the grid's global adds, whose order
# depends on the tiling and varies from run to run, shows in B at that factor: two runs of
# the same member alone differ by up to 8e-6 in B.  B is held to 3e-5, v and F to 1e-5.
TOL_B = 3e-5


def check_same(got, ref, tol=1e-5, tol_B=TOL_B):
    for (gx, gv, gB, gF), (rx, rv, rB, rF) in zip(got, ref):
        assert relerr(gv, rv) <= tol
        assert relerr(gB, rB) <= tol_B
        assert relerr(gF, rF) <= tol
        assert np.abs(gx - rx).max() <= 1e-6


@pytest.mark.parametrize("group", [0, 2, 8])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(apic, use_graph, group):
    """group 0: the component-split P2G (the 3-D default); 2, 8: the cell-parallel one."""
    members = make_members(apic, 6, seed=1)
    steps = 4
    ref = run_alone(apic, members, steps)
    batch = apic.Batch(dim=3, order=2, max_sims=8, max_particles=300000, max_blocks=200000, use_graph=use_graph,
                       group=group)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        batch.add(sim)
        sims.append(sim)
    batch.step(steps)
    st = batch.stats()
    assert st["members"] == 6 and st["steps"] == steps and st["tiles"] > 6
    got = [s.download() for s in sims]
    check_same(got, ref)
    batch.close()


def test_batch_membership_changes(apic):
    """Members leave and join between steps; every simulation still sees exactly its own steps."""
    members = make_members(apic, 5, seed=2)
    ref3 = run_alone(apic, members, 3)
    ref5 = run_alone(apic, members, 5)
    batch = apic.Batch(dim=3, order=2, max_sims=8, max_particles=300000, max_blocks=200000)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        sims.append(sim)
    for s in sims[:3]:
        batch.add(s)
    batch.step(3)
    batch.remove(sims[0])                 # finished after 3 steps
    batch.add(sims[3])                    # joins late
    batch.step(2)
    batch.add(sims[4])
    batch.remove(sims[1])                 # 5 steps
    batch.step(3)                         # sims[2]: 8 steps, sims[3]: 5, sims[4]: 3
    check_same([sims[0].download()], [ref3[0]])
    check_same([sims[1].download()], [ref5[1]])
    check_same([sims[3].download()], [ref5[3]])
    check_same([sims[4].download()], [ref3[4]])
    ref8 = run_alone(apic, members[2:3], 8)
    check_same([sims[2].download()], ref8)
    # a removed simulation can be stepped on its own again
    sims[0].step(2)
    check_same([sims[0].download()], run_alone(apic, members[:1], 5))
    batch.close()


def test_batch_autotune_keeps_results(apic):
    members = make_members(apic, 4, seed=3)
    ref = run_alone(apic, members, 1 + 15 * 2)     # 15 candidates x (1 warm-up + 1 timed) + 1
    batch = apic.Batch(dim=3, order=2, max_sims=4, max_particles=200000, max_blocks=200000)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        batch.add(sim)
        sims.append(sim)
    tile, group = batch.autotune(steps=1, force=True)
    assert tile in (1024, 2048, 4096) and group in (1, 2, 4, 8, apic.APIC_BATCH_SPLIT)
    batch.step(1)
    check_same([s.download() for s in sims], ref)
    batch.close()


def test_batch_2d_fp64(apic):
    members = make_members(apic, 3, seed=4, dim=2, order=3, precision=64, ppc=4)
    ref = run_alone(apic, members, 3)
    batch = apic.Batch(dim=2, order=3, precision=64, max_sims=4, max_particles=200000, max_blocks=200000)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        batch.add(sim)
        sims.append(sim)
    batch.step(3)
    check_same([s.download() for s in sims], ref, tol=1e-11, tol_B=1e-11)
    batch.close()


def test_batch_rejects_incompatible(apic):
    batch = apic.Batch(dim=3, order=2, max_sims=1, max_particles=100000, max_blocks=100000)
    cfg2 = apic.make_config(dim=2, order=2, res=(32, 32), dx=1 / 32)
    s2 = apic.Sim(cfg2, 10)
    s2.upload(np.full((10, 2), 0.5))
    with pytest.raises(apic.ApicError):
        batch.add(s2)
    members = make_members(apic, 2, seed=5)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        sims.append(sim)
    batch.add(sims[0])
    with pytest.raises(apic.ApicError) as e:
        batch.add(sims[1])                # member capacity 1
    assert e.value.status == apic.APIC_ERR_OOM
    with pytest.raises(apic.ApicError):
        sims[0].step(1)                   # members are stepped by the batch only
    batch.close()


def test_batch_fast_motion_equals_alone(apic):
    """Fast rigid rotation in every member, so a large share of the cell keys changes every
    step: the batched sort of the changed keys (several radix tiles per member for the larger
    ones, none at all for the smallest) must reproduce stepping each member alone."""
    rng = np.random.default_rng(21)
    members = []
    for n_target, edge in ((200000, 48), (40000, 32), (3000, 24)):
        res = edge
        side = min(0.5, (n_target / 8) ** (1 / 3) / res)
        sc = scenes.falling_cube_3d(res=res, side=side, ppc=8, seed=int(rng.integers(1 << 30)))
        w = rng.normal(size=3) * 60.0
        v = np.cross(w, sc.x - 0.5)
        vol = sc.dx ** 3 / 8
        cfg = apic.make_config(dim=3, order=2, res=(res,) * 3, dx=sc.dx, dt=1e-4, model="fcr", E=1e4, nu=0.3,
                               particle_mass=vol, particle_volume=vol)
        members.append((cfg, sc.x, v, None, None))
    steps = 4
    ref = run_alone(apic, members, steps)
    batch = apic.Batch(dim=3, order=2, max_sims=4, max_particles=400000, max_blocks=200000)
    sims = []
    for cfg, x, v, B, F in members:
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        batch.add(sim)
        sims.append(sim)
    batch.step(steps)
    check_same([s.download() for s in sims], ref)
    batch.close()


@pytest.mark.parametrize("dim,order,precision", [(3, 2, 32), (3, 3, 32), (2, 3, 64), (2, 2, 32)])
def test_batch_members_match_oracle(apic, dim, order, precision):
    """Every member of a batch against the FP64 oracle, not only against stepping it alone:
    after one batched step, the oracle's step from that member's downloaded input; after two
    more, the oracle's two steps from the state downloaded after the first (each member with
    its own grid, size, material, gravity and walls)."""
    import oracle
    from helpers import configs

    members = make_members(apic, 3, seed=31 + order + dim, dim=dim, order=order, precision=precision,
                           ppc=8 if dim == 3 else 4)
    batch = apic.Batch(dim=dim, order=order, precision=precision, max_sims=4, max_particles=300000,
                       max_blocks=200000)
    sims, inputs, ocfgs = [], [], []
    for i, (cfg, x, v, B, F) in enumerate(members):
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B, F)
        inputs.append(sim.download())                       # the member's exact input state
        res = tuple(cfg.res[a] for a in range(dim))
        g = tuple(cfg.gravity[a] for a in range(dim))
        _, oc, _, _ = configs(dim, order, res, cfg.dx, precision=precision, dt=cfg.dt, gravity=g,
                              boundary="sticky", wall=order + 1, model="fcr", E=cfg.E, nu=cfg.nu)
        ocfgs.append((oc, cfg.particle_mass, cfg.particle_volume))
        batch.add(sim)
        sims.append(sim)
    tol = 1e-5 if precision == 32 else 1e-11
    for nsteps in (1, 2):
        batch.step(nsteps)
        outs = [s.download() for s in sims]
        for i, s in enumerate(sims):
            oc, m, vol = ocfgs[i]
            x0, v0, B0, F0 = inputs[i]
            ox, ov, oB, oF, bad = oracle.step(oc, x0, v0, B0, F0, m, vol, nsteps=nsteps)
            assert bad == 0
            gx, gv, gB, gF = outs[i]
            assert relerr(gv, ov) <= nsteps * tol, f"member {i} after {nsteps} step(s)"
            assert relerr(gB, oB) <= 10 * nsteps * tol, f"member {i}"
            assert relerr(gF, oF) <= nsteps * tol, f"member {i}"
            # the offset in its cell rounds to eps dx; the absolute positions the oracle moves
            # and the download forms round to eps64 |x|
            eps = np.finfo(np.float32 if precision == 32 else np.float64).eps
            bound = nsteps * (tol * np.abs(ox - x0).max() + 2 * eps * oc.dx) + 4 * np.finfo(np.float64).eps
            assert np.abs((gx - x0) - (ox - x0)).max() <= bound, f"member {i}"
        inputs = outs
    batch.close()
