"""Failure detection on the GPU without a GPU fault: the failures are made on the host (a
NaN or Inf in uploaded state) or by a bounded device wait that is told to give up at once
(the library's wait-limit hook); each must come back as an error code while the device
stays usable for the next simulation."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, relerr
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


def cube_state(seed=0):
    sc = scenes.falling_cube_3d(res=32, side=0.5, ppc=8, seed=seed, omega=(0.0, 0.0, 1.0))
    B = sc.grad_v * kappa(2) * sc.dx ** 2
    F = scenes.random_deformation(np.random.default_rng(seed), sc.n, 3, 0.05)
    return sc, sc.x.copy(), sc.v.copy(), B, F


def one_step_matches_oracle(apic, sc, x, v, B, F):
    gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4)
    sim = apic.Sim(gc, len(x))
    sim.upload(x, v, B, F)
    x0, v0, B0, F0 = sim.download()
    sim.step(1)
    gx, gv, gB, gF = sim.download()
    ox, ov, oB, oF, bad = oracle.step(oc, x0, v0, B0, F0, m, vol)
    sim.close()
    return bad == 0 and relerr(gv, ov) <= 1e-5 and relerr(gB, oB) <= 1e-5 and relerr(gF, oF) <= 1e-5


@pytest.mark.parametrize("field,value", [("x", np.nan), ("v", np.inf), ("B", -np.inf), ("F", np.nan)])
def test_nonfinite_host_upload_is_rejected(apic, field, value):
    sc, x, v, B, F = cube_state()
    arrs = {"x": x, "v": v, "B": B, "F": F}
    arrs[field] = arrs[field].copy()
    arrs[field].reshape(len(x), -1)[len(x) // 2, 0] = value
    gc, _, _, _ = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4)
    sim = apic.Sim(gc, len(x))
    with pytest.raises(apic.ApicError) as e:
        sim.upload(arrs["x"], arrs["v"], arrs["B"], arrs["F"])
    assert e.value.status == apic.APIC_ERR_NUMERIC
    assert "non-finite" in str(e.value)
    assert sim.n == 0 and sim.stats()["particles"] == 0    # the upload was discarded
    # the same simulation takes a clean upload afterwards and steps like the oracle
    sim.upload(x, v, B, F)
    sim.step(1)
    sim.download()
    sim.close()


def test_nonfinite_device_upload_is_reported_at_the_next_synchronising_call(apic):
    torch = pytest.importorskip("torch")
    sc, x, v_clean, B, F = cube_state(1)
    v = v_clean.copy()
    v[7, 2] = np.nan
    gc, _, _, _ = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4)
    sim = apic.Sim(gc, len(x))
    sim.upload(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, v, B, F)))
    with pytest.raises(apic.ApicError) as e:
        sim.download()
    assert e.value.status == apic.APIC_ERR_NUMERIC
    sim.close()
    assert one_step_matches_oracle(apic, sc, x, v_clean, B, F)


def test_bounded_wait_runs_out_and_reports_timeout(apic):
    """G2P's first wait for its staged grid blocks is told to give up without polling: every
    CTA latches the timeout, lets its copies land and leaves; the next synchronising call
    returns APIC_ERR_TIMEOUT and the next simulation on the device steps correctly."""
    sc, x, v, B, F = cube_state(2)
    gc, _, _, _ = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4)
    sim = apic.Sim(gc, len(x))
    sim.upload(x, v, B, F)
    apic.apic_set_wait_limit(sim.handle, 0)
    sim.step(1)
    # a reduction over the state (no indexed writes) is the synchronising call that reads
    # the latched word; the state of this step is not valid
    with pytest.raises(apic.ApicError) as e:
        sim.momentum("particles")
    assert e.value.status == apic.APIC_ERR_TIMEOUT
    sim.close()
    assert one_step_matches_oracle(apic, sc, x, v, B, F)


def test_default_wait_limit_does_not_trip(apic):
    sc, x, v, B, F = cube_state(3)
    gc, _, _, _ = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4)
    sim = apic.Sim(gc, len(x))
    sim.upload(x, v, B, F)
    apic.apic_set_wait_limit(sim.handle, 1 << 22)
    sim.step(3)
    sim.download()
    sim.close()
