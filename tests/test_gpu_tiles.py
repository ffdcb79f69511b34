"""The tile list that P2G and G2P walk: a tile is a maximal run of sorted particles with the
same node block inside one aligned chunk of tile_particles particles, so a new tile starts at
every chunk start and at every change of block.  The GPU's tile count after each sort must
equal that rule applied on the host to the downloaded sorted keys, for every tile size, in
2-D and 3-D, with a ragged last chunk, after the full sort and after incremental sorts."""
import numpy as np
import pytest

from helpers import configs, state_for
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


def host_tile_count(keys: np.ndarray, dim: int, tile: int) -> int:
    blk = keys.astype(np.int64) >> (2 * dim)
    idx = np.arange(len(keys))
    head = idx % tile == 0
    head[1:] |= blk[1:] != blk[:-1]
    return int(np.count_nonzero(head))


@pytest.mark.parametrize("tile", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("dim", [2, 3])
def test_tile_count_matches_rule(apic, tile, dim):
    if dim == 3:
        sc = scenes.falling_cube_3d(res=40, side=0.45, ppc=8, omega=(0.0, 0.0, 30.0), seed=5)
        res = (40,) * 3
    else:
        sc = scenes.rotating_disk_2d(res=160, radius=0.3, ppc=4, seed=5, omega=30.0)
        res = (160,) * 2
    assert sc.n % tile != 0   # a ragged last chunk
    x, v, B, F = state_for(sc, 2, seed=5)
    gc, _, m, vol = configs(dim, 2, res, sc.dx, dt=2e-4, tile=tile, boundary="sticky", wall=3)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    for step in range(4):   # the full sort, then incremental ones
        sim.p2g()
        keys, _ = sim.keys()
        assert np.all(keys[1:] >= keys[:-1])
        assert sim.stats()["tiles"] == host_tile_count(keys, dim, tile), f"step {step}"
        sim.grid_update()
        sim.g2p()
    sim.close()


def test_tile_list_through_the_chunk_scan(apic):
    """More than 4096 chunks of 256 particles: the chunk offsets come from the device scan
    instead of the per-chunk reduction; the list must still satisfy the rule, and one step
    through it must give the same grid and particles as with 4096-particle tiles (one chunk
    per block there, the reduction path)."""
    sc = scenes.falling_cube_3d(res=128, side=0.45, ppc=8, omega=(0.0, 0.0, 20.0), seed=7)
    assert (sc.n + 255) // 256 > 4096
    x, v, B, F = state_for(sc, 2, seed=7)
    out = []
    for tile in (256, 4096):
        gc, _, _, _ = configs(3, 2, (128,) * 3, sc.dx, dt=2e-4, tile=tile, boundary="sticky", wall=3)
        sim = apic.Sim(gc, sc.n)
        sim.upload(x, v, B, F)
        for step in range(3):
            sim.p2g()
            keys, _ = sim.keys()
            assert sim.stats()["tiles"] == host_tile_count(keys, 3, tile), f"tile {tile}, step {step}"
            sim.grid_update()
            sim.g2p()
        out.append(sim.download())
        sim.close()
    # the same arithmetic; the two tilings differ only in the order of the grid's global adds
    # (B, a small difference of larger terms under the rotation, is held to 3e-5 as in the
    # batch tests)
    for a, b, tol in zip(*out, (1e-5, 1e-5, 3e-5, 1e-5)):
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-30)
