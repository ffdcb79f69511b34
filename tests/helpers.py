"""Shared helpers of the test suite: seeded states, oracle/GPU config pairs, error norms."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1603_06188_gb300 import scenes

E_DEFAULT, NU_DEFAULT = 1e4, 0.3


def kappa(order: int) -> float:
    """D_p = kappa dx^2 I for B-splines (the constants Sec. 5.6 prints)."""
    return 0.25 if order == 2 else 1.0 / 3.0


def relerr(got, ref) -> float:
    """Normwise relative error ||got - ref||_inf / ||ref||_inf."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max() if ref.size else 0.0
    if den == 0.0:
        return float(np.abs(got).max()) if got.size else 0.0
    return float(np.abs(got - ref).max() / den)


def state_for(scene: scenes.Scene, order: int, seed: int = 0, vscale: float = 1.0, Bscale: float = 1.0,
              Fscale: float = 0.1):
    """Particles of a scene with rigid velocity, affine B = grad_v D_p plus seeded noise in
    v, B and F so every term of the transfers is exercised."""
    rng = np.random.default_rng(seed)
    n, d = scene.n, scene.dim
    k = kappa(order) * scene.dx ** 2
    v = scene.v * vscale + 0.1 * rng.normal(size=(n, d))
    B = Bscale * (scene.grad_v * k + 0.05 * k / scene.dx * rng.normal(size=(n, d, d)))
    F = scenes.random_deformation(rng, n, d, Fscale)
    return scene.x.copy(), v, B, F


def configs(dim, order, res, dx, precision=32, transfer="apic", dt=1e-3, gravity=(0, 0, 0),
            boundary="none", wall=0, model="fcr", E=E_DEFAULT, nu=NU_DEFAULT, mass=1.0, vol=None,
            tile=0, p2g_kernel=0, p2g_group=0):
    """Matching (library config, oracle config, mass, volume)."""
    from paper_1603_06188_gb300 import apic

    if vol is None:
        vol = dx ** dim / 8
    gc = apic.make_config(dim=dim, order=order, precision=precision, transfer=transfer, res=res, dx=dx, dt=dt,
                          gravity=gravity, boundary=boundary, wall=wall, model=model, E=E, nu=nu,
                          particle_mass=mass, particle_volume=vol, tile_particles=tile, p2g_kernel=p2g_kernel,
                          p2g_group=p2g_group)
    oc = oracle.make_cfg(dim=dim, order=order, transfer=transfer, res=res, dx=dx, dt=dt, gravity=gravity,
                         boundary=boundary, wall=wall,
                         model={"fcr": "fcr", "fixed_corotated": "fcr", "nh": "nh", "neohookean": "nh"}.get(model, "none"),
                         E=E, nu=nu)
    return gc, oc, mass, vol


def occupancy_rule(keys: np.ndarray, dim: int, res) -> np.ndarray:
    """Active node blocks of the block-sparse grid: every particle's stencil-base block b
    plus b + {0,1}^dim (the blocks its stencil can reach), inside the grid."""
    nb = [(r + 3) // 4 for r in res[:dim]]
    out = np.zeros(int(np.prod(nb)), dtype=np.uint8)
    blk = (keys.astype(np.int64) >> (2 * dim))
    coords = []
    r = blk.copy()
    for a in range(dim):
        coords.append(r % nb[a])
        r //= nb[a]
    for delta in range(1 << dim):
        ok = np.ones(len(blk), dtype=bool)
        lin = np.zeros(len(blk), dtype=np.int64)
        mult = 1
        for a in range(dim):
            c = coords[a] + ((delta >> a) & 1)
            ok &= c < nb[a]
            lin += c * mult
            mult *= nb[a]
        out[lin[ok]] = 1
    return out


def nodewise_err(got, ref, mass, floor: float = 0.1) -> float:
    """Largest error at any grid node relative to that node's own scale: the largest of
    |ref_i|, the node's share of the mass times the largest |ref|, and `floor` times the
    largest |ref| (so with a bound tol, a node with little mass must be within tol * floor of
    the largest value, `1 / floor` times tighter than the normwise bound; the floor covers
    nodes reached only by weights close to zero, which FP32 resolves to a few ulps of the
    largest weight).  Nodes whose scale is zero must be exactly zero."""
    got = np.asarray(got, dtype=np.float64).reshape(len(mass), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(mass), -1)
    mass = np.asarray(mass, dtype=np.float64)
    big = np.abs(ref).max() if ref.size else 0.0
    mmax = mass.max() if mass.size else 0.0
    share = mass / mmax if mmax > 0 else np.zeros_like(mass)
    scale = np.maximum(np.maximum(np.abs(ref).max(axis=1), share * big), floor * big)
    err = np.abs(got - ref).max(axis=1)
    zero = scale == 0.0
    if np.any(err[zero] != 0.0):
        return float("inf")
    return float((err[~zero] / scale[~zero]).max()) if np.any(~zero) else 0.0


def stencil_max_speed(x, gv, res, dx, order) -> np.ndarray:
    """Per particle, the largest |v~_i| over the nodes of its B-spline stencil (dense grid
    velocities gv of shape (nodes, d), node index i0 + N0 (i1 + N1 i2))."""
    x = np.asarray(x, dtype=np.float64)
    n, d = x.shape
    u = x / dx
    base = np.floor(u - 0.5).astype(np.int64) if order == 2 else np.floor(u).astype(np.int64) - 1
    speed = np.sqrt((np.asarray(gv) ** 2).sum(axis=1))
    out = np.zeros(n)
    k = order + 1
    for off in np.ndindex(*([k] * d)):
        idx = np.zeros(n, dtype=np.int64)
        mult = 1
        ok = np.ones(n, dtype=bool)
        for a in range(d):
            g = base[:, a] + off[a]
            ok &= (g >= 0) & (g < res[a])
            idx += np.clip(g, 0, res[a] - 1) * mult
            mult *= res[a]
        out = np.maximum(out, np.where(ok, speed[idx], 0.0))
    return out


def particlewise_err(got, ref, scale) -> float:
    """Largest error of any particle's entries relative to that particle's own scale."""
    got = np.asarray(got, dtype=np.float64).reshape(len(scale), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(scale), -1)
    scale = np.asarray(scale, dtype=np.float64)
    err = np.abs(got - ref).max(axis=1)
    zero = scale == 0.0
    if np.any(err[zero] != 0.0):
        return float("inf")
    return float((err[~zero] / scale[~zero]).max()) if np.any(~zero) else 0.0
