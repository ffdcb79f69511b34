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
        assert relerr(gB, aB) <= 1e-5
        assert relerr(gF, aF) <= 1e-5
        assert np.abs(gx - ax).max() <= 1e-6
        sim.close()
    batch.close()
