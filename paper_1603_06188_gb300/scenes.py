"""Seeded synthetic scenes shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds no part of the APIC method's arithmetic: it only places particles in
simple shapes and gives them initial rigid-body velocities.  Every scene is a pure
function of its arguments and its seed (numpy PCG64).

Sampling ("jittered uniform"): each grid cell inside the shape's bounding box is split
into ``ppc`` equal sub-cells (2x2 for 4 ppc in 2-D, 2x2x2 for 8 ppc, 4x4x2 for 32 ppc in
3-D) and one uniform point is drawn in each sub-cell; points outside the shape are
dropped.  Velocities are rigid: ``v = v0 + omega x (x - c)``; ``grad_v`` is the
corresponding constant velocity-gradient matrix (a skew matrix), so a caller that wants
an affine initial state sets ``B_p = grad_v D_p``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _subdiv(dim: int, ppc: int) -> tuple[int, ...]:
    table = {(2, 1): (1, 1), (2, 4): (2, 2), (2, 9): (3, 3), (2, 16): (4, 4),
             (3, 1): (1, 1, 1), (3, 8): (2, 2, 2), (3, 27): (3, 3, 3), (3, 32): (4, 4, 2),
             (3, 64): (4, 4, 4)}
    if (dim, ppc) not in table:
        raise ValueError(f"unsupported particles-per-cell {ppc} in {dim}-D")
    return table[(dim, ppc)]


def _skew(omega, dim: int) -> np.ndarray:
    if dim == 2:
        w = float(np.asarray(omega).reshape(-1)[0])
        return np.array([[0.0, -w], [w, 0.0]])
    wx, wy, wz = (float(t) for t in omega)
    return np.array([[0.0, -wz, wy], [wz, 0.0, -wx], [-wy, wx, 0.0]])


@dataclass
class Body:
    """Particles of one body: positions (n, d), velocities (n, d), grad_v (d, d)."""

    x: np.ndarray
    v: np.ndarray
    grad_v: np.ndarray


@dataclass
class Scene:
    dim: int
    res: tuple[int, ...]
    dx: float
    ppc: int
    x: np.ndarray
    v: np.ndarray
    grad_v: np.ndarray          # (n, d, d): per-particle velocity gradient of the rigid motion
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.x)


def sample_shape(rng: np.random.Generator, dim: int, dx: float, ppc: int, lo, hi, inside) -> np.ndarray:
    """Stratified jittered points in the cells covering [lo, hi], filtered by ``inside``."""
    sub = np.array(_subdiv(dim, ppc))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c0 = np.floor(lo / dx).astype(np.int64)
    c1 = np.ceil(hi / dx).astype(np.int64)
    axes = [np.arange(c0[a], c1[a]) for a in range(dim)]
    cells = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    subs = np.stack(np.meshgrid(*[np.arange(s) for s in sub], indexing="ij"), axis=-1).reshape(-1, dim)
    # every (cell, sub-cell) pair gets one uniform point inside that sub-cell
    base = (cells[:, None, :] + subs[None, :, :] / sub).reshape(-1, dim)
    jit = rng.random(base.shape) / sub
    pts = (base + jit) * dx
    keep = inside(pts)
    return pts[keep]


def rigid_velocity(x: np.ndarray, center, v0, omega) -> tuple[np.ndarray, np.ndarray]:
    dim = x.shape[1]
    W = _skew(omega, dim)
    v = np.asarray(v0, dtype=np.float64)[None, :] + (x - np.asarray(center)[None, :]) @ W.T
    return v, W


def ball(rng, dim, dx, ppc, center, radius, v0, omega) -> Body:
    c = np.asarray(center, dtype=np.float64)
    x = sample_shape(rng, dim, dx, ppc, c - radius, c + radius,
                     lambda p: np.sum((p - c) ** 2, axis=1) < radius * radius)
    v, W = rigid_velocity(x, c, v0, omega)
    return Body(x, v, W)


def box(rng, dim, dx, ppc, lo, hi, v0, omega) -> Body:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x = sample_shape(rng, dim, dx, ppc, lo, hi, lambda p: np.all((p >= lo) & (p < hi), axis=1))
    v, W = rigid_velocity(x, 0.5 * (lo + hi), v0, omega)
    return Body(x, v, W)


def _scene(dim, res, dx, ppc, bodies, **meta) -> Scene:
    x = np.concatenate([b.x for b in bodies])
    v = np.concatenate([b.v for b in bodies])
    gv = np.concatenate([np.broadcast_to(b.grad_v, (len(b.x), dim, dim)) for b in bodies])
    return Scene(dim, tuple(res), dx, ppc, x, v, np.ascontiguousarray(gv), meta)


def rotating_disk_2d(res: int = 64, radius: float = 0.3, center=(0.5, 0.5), ppc: int = 4,
                     omega: float = 1.0, v0=(0.1, 0.0), seed: int = 0) -> Scene:
    """2-D disk in rigid rotation plus translation (shape of the paper's Sec. 6.1 test)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    b = ball(rng, 2, dx, ppc, center, radius, v0, [omega])
    return _scene(2, (res, res), dx, ppc, [b], kind="rotating_disk_2d", seed=seed)


def falling_cube_3d(res: int = 128, side: float = 0.4, center=(0.5, 0.5, 0.5), ppc: int = 8,
                    v0=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), seed: int = 0) -> Scene:
    """3-D elastic cube (centred, at rest unless v0 / omega given)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    c = np.asarray(center, dtype=np.float64)
    b = box(rng, 3, dx, ppc, c - side / 2, c + side / 2, v0, omega)
    return _scene(3, (res, res, res), dx, ppc, [b], kind="falling_cube_3d", seed=seed)


def colliding_spheres_3d(res: int = 256, radius: float = 0.15, ppc: int = 8, speed: float = 1.0,
                         centers=((0.345, 0.5, 0.5), (0.655, 0.5, 0.5)), omega=(0.0, 0.0, 0.0),
                         seed: int = 0) -> Scene:
    """Two 3-D spheres approaching along x (shape of the paper's Sec. 6.5 collision)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    b1 = ball(rng, 3, dx, ppc, centers[0], radius, (speed, 0.0, 0.0), omega)
    b2 = ball(rng, 3, dx, ppc, centers[1], radius, (-speed, 0.0, 0.0), omega)
    return _scene(3, (res, res, res), dx, ppc, [b1, b2], kind="colliding_spheres_3d", seed=seed)


def random_sim_spec(rng: np.random.Generator, edge_range=(32, 96), np_range=(2_000, 400_000)) -> dict:
    """One simulation of the batched mix: grid edge uniform, particle count log-uniform."""
    edge = int(rng.integers(edge_range[0], edge_range[1] + 1))
    target = float(np.exp(rng.uniform(np.log(np_range[0]), np.log(np_range[1]))))
    shape = "box" if rng.random() < 0.5 else "sphere"
    v0 = rng.uniform(-0.5, 0.5, size=3)
    omega = rng.uniform(-2.0, 2.0, size=3)
    return {"edge": edge, "target_particles": target, "shape": shape, "v0": v0, "omega": omega,
            "seed": int(rng.integers(0, 2**31 - 1))}


def sim_from_spec(spec: dict, ppc: int = 8, margin_cells: int = 6) -> Scene:
    """Build the particles of one batched simulation from ``random_sim_spec``.

    The body's volume is chosen so that ``ppc`` particles per cell give about the target
    count, clamped to the interior of the grid (a margin of ``margin_cells`` cells).
    """
    edge = spec["edge"]
    dx = 1.0 / edge
    rng = np.random.default_rng(spec["seed"])
    cells = spec["target_particles"] / ppc
    room = 1.0 - 2.0 * margin_cells * dx
    if spec["shape"] == "box":
        side = min(cells ** (1.0 / 3.0) * dx, room)
        c = np.full(3, 0.5)
        b = box(rng, 3, dx, ppc, c - side / 2, c + side / 2, spec["v0"], spec["omega"])
    else:
        r = min((cells * 3.0 / (4.0 * np.pi)) ** (1.0 / 3.0) * dx, room / 2)
        b = ball(rng, 3, dx, ppc, np.full(3, 0.5), r, spec["v0"], spec["omega"])
    return _scene(3, (edge, edge, edge), dx, ppc, [b], kind=f"batched_{spec['shape']}", seed=spec["seed"])


def random_deformation(rng: np.random.Generator, n: int, dim: int, scale: float = 0.1) -> np.ndarray:
    """Deformation gradients F = I + scale * U(-1, 1) entries (positive determinant for small scale)."""
    return np.eye(dim)[None, :, :] + scale * rng.uniform(-1.0, 1.0, size=(n, dim, dim))


def random_particles(rng: np.random.Generator, n: int, dim: int, res, dx: float, margin: int = 4):
    """Uniform random positions inside the grid (keeping ``margin`` nodes from each face)."""
    res = np.asarray(res)
    lo = margin * dx
    hi = (res[:dim] - 1 - margin) * dx
    return lo + rng.random((n, dim)) * (hi - lo)
