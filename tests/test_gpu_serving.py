"""Serving on the GPU: requests arrive while others run, are admitted under a memory budget
and leave when done; each one's final state must equal running it alone for its steps."""
import numpy as np
import pytest

from helpers import kappa, relerr
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic, serving

    apic.load(build_if_missing=True)
    rng = np.random.default_rng(21)
    reqs, payloads = [], {}
    arrivals = serving.poisson_arrivals(rng, 500.0, 7)
    for i in range(7):
        spec = scenes.random_sim_spec(rng, edge_range=(24, 36), np_range=(2000, 20000))
        sc = scenes.sim_from_spec(spec, ppc=8)
        vol = sc.dx ** 3 / 8
        cfg = apic.make_config(dim=3, order=2, res=sc.res, dx=sc.dx, dt=2e-5, gravity=(0.0, -9.8, 0.0),
                               boundary="sticky", wall=3, model="fcr", E=1e4, nu=0.3, particle_mass=vol,
                               particle_volume=vol)
        B = sc.grad_v * kappa(2) * sc.dx ** 2
        steps = int(rng.integers(3, 12))
        payloads[i] = (cfg, sc.x, sc.v, B)
        reqs.append(serving.Request(i, float(arrivals[i]), steps, apic.apic_workspace_size(cfg, sc.n), sc.n))
    budget = sum(sorted(r.footprint for r in reqs)[-3:])          # at most ~3 resident: forces queueing
    batch = apic.Batch(dim=3, order=2, max_sims=8, max_particles=200000, max_blocks=200000)

    def make_sim(r):
        cfg, x, v, B = payloads[r.rid]
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B)
        return sim

    rep, results = serving.serve_gpu(reqs, make_sim, batch, budget, max_resident=8, max_chunk=2, keep_state=True)
    assert rep.completed == 7 and rep.max_bytes <= budget
    assert rep.max_resident >= 2
    for r in reqs:
        cfg, x, v, B = payloads[r.rid]
        sim = apic.Sim(cfg, len(x))
        sim.upload(x, v, B)
        sim.step(r.steps)
        ax, av, aB, aF = sim.download()
        gx, gv, gB, gF = results[r.rid]
        assert relerr(gv, av) <= 1e-5
        assert relerr(gB, aB) <= 3e-5   # B rounding under rigid motion, as in test_gpu_batch
        assert relerr(gF, aF) <= 1e-5
        assert np.abs(gx - ax).max() <= 1e-6
        sim.close()
    batch.close()


def test_batch_admit_and_run_through_the_c_abi():
    """apic_batch_admit refuses a member whose footprint would take the admitted total over
    the budget (APIC_ERR_OOM, nothing changes) and admits it once a completion frees room;
    apic_batch_run never steps past the nearest completion, hands back exactly the members
    whose steps are done (in membership order) and frees their bytes; each finished member
    equals the same simulation stepped alone for its steps."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic

    apic.load(build_if_missing=True)
    rng = np.random.default_rng(5)
    payloads = []
    for i in range(4):
        spec = scenes.random_sim_spec(rng, edge_range=(24, 32), np_range=(3000, 12000))
        sc = scenes.sim_from_spec(spec, ppc=8)
        vol = sc.dx ** 3 / 8
        cfg = apic.make_config(dim=3, order=2, res=sc.res, dx=sc.dx, dt=2e-5, model="fcr", E=1e4, nu=0.3,
                               particle_mass=vol, particle_volume=vol)
        payloads.append((cfg, sc.x, sc.v, sc.grad_v * kappa(2) * sc.dx ** 2))
    steps = [5, 3, 7, 4]
    foot = [1000, 2000, 3000, 1500]
    budget = 5500
    batch = apic.Batch(dim=3, order=2, max_sims=8, max_particles=200000, max_blocks=200000)
    sims = []
    for cfg, x, v, B in payloads:
        s = apic.Sim(cfg, len(x))
        s.upload(x, v, B)
        sims.append(s)
    batch.admit(sims[0], steps[0], foot[0], budget)
    batch.admit(sims[1], steps[1], foot[1], budget)
    assert batch.resident_bytes() == 3000
    with pytest.raises(apic.ApicError) as e:
        batch.admit(sims[2], steps[2], foot[2], budget)          # 3000 + 3000 > 5500
    assert e.value.status == apic.APIC_ERR_OOM
    assert batch.resident_bytes() == 3000 and len(batch.members) == 2
    batch.admit(sims[3], steps[3], foot[3], budget)               # 4500 <= 5500
    fin, k = batch.run(8)
    assert k == 3 and fin == [sims[1]]                            # the nearest completion: 3 steps
    assert batch.resident_bytes() == 2500
    batch.admit(sims[2], steps[2], foot[2], budget)               # 2500 + 3000 <= 5500 now
    fin, k = batch.run(8)
    assert k == 1 and fin == [sims[3]]                            # sims[3] had 4 - 3 = 1 left
    fin, k = batch.run(8)
    assert k == 1 and fin == [sims[0]]                            # sims[0]: 5 - 3 - 1 = 1 left
    fin, k = batch.run(2)
    assert k == 2 and fin == []                                   # capped by max_steps
    fin, k = batch.run(8)
    assert k == 3 and fin == [sims[2]] and batch.resident_bytes() == 0   # 1 + 1 + 2 + 3 = 7
    assert batch.members == []
    done_steps = dict(enumerate(steps))
    for i, (cfg, x, v, B) in enumerate(payloads):
        alone = apic.Sim(cfg, len(x))
        alone.upload(x, v, B)
        alone.step(done_steps[i])
        ax, av, aB, aF = alone.download()
        gx, gv, gB, gF = sims[i].download()
        assert relerr(gv, av) <= 1e-5
        assert relerr(gB, aB) <= 3e-5   # B rounding under rigid motion, as in test_gpu_batch
        assert relerr(gF, aF) <= 1e-5
        assert np.abs(gx - ax).max() <= 1e-6
        alone.close()
    batch.close()
