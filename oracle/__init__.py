"""FP64 CPU oracle for the APIC / explicit MPM step (arXiv:1603.06188).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the CUDA path is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import it; the product package never does.  It shares no code with
the CUDA library: the C source here is compiled on its own with gcc and called through
ctypes with numpy arrays.

Each wrapper names the part of the paper it follows; the C file holds the arithmetic.
Array conventions: positions / velocities ``(n, d)``, matrices ``(n, d, d)`` row-major,
dense grids ``(N_{d-1}, ..., N_0)`` flattened with axis 0 fastest (node ``i0 + N0*(i1 +
N1*i2)``), grid vectors ``(nodes, d)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain -O2, no fast-math) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(C.Structure):
    """Mirror of ``or_cfg`` in apic_oracle.c."""

    _fields_ = [
        ("dim", C.c_int), ("order", C.c_int), ("transfer", C.c_int),
        ("res", C.c_int * 3), ("dx", C.c_double), ("origin", C.c_double * 3),
        ("dt", C.c_double), ("gravity", C.c_double * 3),
        ("boundary", C.c_int), ("wall", C.c_int), ("model", C.c_int),
        ("mu", C.c_double), ("lam", C.c_double), ("lambda_t", C.c_double), ("flip_alpha", C.c_double),
    ]


def lame(E: float, nu: float) -> tuple[float, float]:
    """Lame parameters mu, lambda from Young's modulus and Poisson's ratio."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def make_cfg(dim=3, order=2, transfer="apic", res=(16, 16, 16), dx=1.0 / 16, origin=(0, 0, 0),
             dt=0.0, gravity=(0, 0, 0), boundary="none", wall=0, model="none", E=0.0, nu=0.0,
             lambda_t=0.0, flip_alpha=1.0) -> Cfg:
    """transfer: "apic", "pic" or "flip" (a PIC/FLIP blend with weight flip_alpha on FLIP)."""
    c = Cfg()
    c.dim, c.order = dim, order
    c.transfer = {"apic": 0, "pic": 1, "flip": 2}[transfer]
    c.flip_alpha = flip_alpha
    r = list(res) + [1] * (3 - len(res))
    c.res = (C.c_int * 3)(*r)
    c.dx = dx
    o = list(origin) + [0.0] * (3 - len(origin))
    c.origin = (C.c_double * 3)(*o)
    c.dt = dt
    g = list(gravity) + [0.0] * (3 - len(gravity))
    c.gravity = (C.c_double * 3)(*g)
    c.boundary = {"none": 0, "sticky": 1, "slip": 2}[boundary]
    c.wall = wall
    c.model = {"none": 0, "fcr": 1, "nh": 2}[model]
    if model in ("fcr", "nh"):
        c.mu, c.lam = lame(E, nu)
    c.lambda_t = lambda_t
    return c


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, cp = C.c_double, C.c_int64, C.c_void_p
            cfgp = C.POINTER(Cfg)
            sig = {
                "or_N": (d, [C.c_int, d]),
                "or_dN": (d, [C.c_int, d]),
                "or_stencil": (C.c_int, [cfgp, cp, cp, cp, cp]),
                "or_weights_all": (None, [cfgp, cp, cp, cp]),
                "or_svd": (None, [C.c_int, cp, cp, cp, cp]),
                "or_polar": (None, [C.c_int, cp, cp]),
                "or_psi_fcr": (d, [C.c_int, d, d, cp]),
                "or_stress_fcr": (None, [C.c_int, d, d, cp, cp]),
                "or_psi_nh": (d, [C.c_int, d, d, cp]),
                "or_stress_nh": (None, [C.c_int, d, d, cp, cp]),
                "or_cfl_speed": (d, [cfgp, i64, cp, cp]),
                "or_p2g": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp, cp, cp, cp]),
                "or_p2g_mat": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp, cp, cp, cp, cp, cp]),
                "or_step_mat": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp, cp, cp]),
                "or_grid_update": (None, [cfgp, cp, cp, cp, cp, cp]),
                "or_g2p": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp]),
                "or_g2p_lambda0": (i64, [cfgp, i64, cp, cp, cp, cp, cp]),
                "or_potential": (d, [cfgp, i64, cp, cp, cp, cp]),
                "or_force_at": (i64, [cfgp, i64, cp, cp, cp, cp, cp]),
                "or_step_lambda1": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp]),
                "or_dstress_fcr": (None, [C.c_int, d, d, cp, cp, cp]),
                "or_dstress_nh": (None, [C.c_int, d, d, cp, cp, cp]),
                "or_force_diff_at": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp]),
                "or_step_midpoint": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp, C.c_int, C.c_int, d]),
                "or_midpoint_solve": (C.c_int, [cfgp, i64, cp, cp, cp, cp, cp, C.c_int, C.c_int, d, cp]),
                "or_momentum_particles": (None, [cfgp, i64, cp, cp, cp, cp, cp, cp]),
                "or_momentum_grid": (None, [cfgp, cp, cp, cp]),
                "or_keys": (None, [cfgp, C.c_int, i64, cp, cp, cp]),
                "or_stable_sort": (None, [i64, cp, cp]),
                "or_step": (i64, [cfgp, i64, cp, cp, cp, cp, cp, cp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _nodes(cfg: Cfg) -> int:
    n = 1
    for a in range(cfg.dim):
        n *= cfg.res[a]
    return n


# --------------------------------------------------------------------------- weights
def N(order: int, t: float) -> float:
    """1-D cardinal B-spline of the given order (Sec. 3.5 interpolation kernel)."""
    return _load().or_N(order, float(t))


def dN(order: int, t: float) -> float:
    return _load().or_dN(order, float(t))


def stencil(cfg: Cfg, xp):
    """Base node, weights w_ip and gradients grad w_ip of one particle (Sec. 3.5)."""
    d, K = cfg.dim, cfg.order + 1
    xp = _f64(xp)
    base = np.zeros(3, dtype=np.int32)
    w = np.zeros(K ** d)
    dw = np.zeros((K ** d, d))
    rc = _load().or_stencil(C.byref(cfg), _p(xp), _p(base), _p(w), _p(dw))
    return rc, base[:d].copy(), w, dw


def stencil_nodes(cfg: Cfg, base) -> np.ndarray:
    """Node coordinates x_i of the stencil nodes in the oracle's order, shape (K^d, d)."""
    d, K = cfg.dim, cfg.order + 1
    out = np.zeros((K ** d, d))
    for j in range(K ** d):
        r = j
        for a in range(d):
            out[j, a] = cfg.origin[a] + (base[a] + r % K) * cfg.dx
            r //= K
    return out


def weights_all(cfg: Cfg, xp):
    """Brute-force w_ip, grad w_ip over every node of the grid (Sec. 3.5 definition)."""
    nn = _nodes(cfg)
    w = np.zeros(nn)
    dw = np.zeros((nn, cfg.dim))
    _load().or_weights_all(C.byref(cfg), _p(_f64(xp)), _p(w), _p(dw))
    return w, dw


# --------------------------------------------------------------------------- stress
def svd(F):
    F = _f64(F)
    d = F.shape[0]
    U = np.zeros((d, d)); s = np.zeros(d); V = np.zeros((d, d))
    _load().or_svd(d, _p(F), _p(U), _p(s), _p(V))
    return U, s, V


def polar(F):
    F = _f64(F)
    d = F.shape[0]
    R = np.zeros((d, d))
    _load().or_polar(d, _p(F), _p(R))
    return R


def psi_fcr(F, mu, lam) -> float:
    F = _f64(F)
    return _load().or_psi_fcr(F.shape[0], mu, lam, _p(F))


def stress_fcr(F, mu, lam):
    F = _f64(F)
    P = np.zeros_like(F)
    _load().or_stress_fcr(F.shape[0], mu, lam, _p(F), _p(P))
    return P


def psi_nh(F, mu, lam) -> float:
    F = _f64(F)
    return _load().or_psi_nh(F.shape[0], mu, lam, _p(F))


def stress_nh(F, mu, lam):
    F = _f64(F)
    P = np.zeros_like(F)
    _load().or_stress_nh(F.shape[0], mu, lam, _p(F), _p(P))
    return P


def cfl_speed(cfg: Cfg, v, B) -> float:
    """max_p (|v_p| + (kappa/k) dx |B_p|_F) of Sec. 4.3; dt <= nu dx / this."""
    d = cfg.dim
    n = len(v)
    return _load().or_cfl_speed(C.byref(cfg), n, _p(_f64(v, (n, d))), _p(_f64(B, (n, d, d))))


# --------------------------------------------------------------------------- transfers
def p2g(cfg: Cfg, x, v, B, F, mass, vol, mu=None, lam=None):
    """Sec. 3.2 transfer to grid plus the Sec. 3.3 force.  Returns (m, mv, f, n_skipped).
    mu, lam: per-particle Lame parameters (a material per particle); None = the config's."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)); v = _f64(v, (n, d)); B = _f64(B, (n, d, d)); F = _f64(F, (n, d, d))
    mass = _f64(np.broadcast_to(mass, (n,))); vol = _f64(np.broadcast_to(vol, (n,)))
    nn = _nodes(cfg)
    gm = np.zeros(nn); gmv = np.zeros((nn, d)); gf = np.zeros((nn, d))
    if mu is None:
        bad = _load().or_p2g(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol),
                             _p(gm), _p(gmv), _p(gf))
    else:
        mu = _f64(np.broadcast_to(mu, (n,))); lam = _f64(np.broadcast_to(lam, (n,)))
        bad = _load().or_p2g_mat(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol), _p(mu),
                                 _p(lam), _p(gm), _p(gmv), _p(gf))
    return gm, gmv, gf, bad


def grid_update(cfg: Cfg, gm, gmv, gf):
    """Sec. 3.3 explicit grid update (lambda = 0).  Returns (v, v~)."""
    d = cfg.dim
    nn = _nodes(cfg)
    gm = _f64(gm); gmv = _f64(gmv, (nn, d)); gf = _f64(gf, (nn, d))
    gv = np.zeros((nn, d)); gvt = np.zeros((nn, d))
    _load().or_grid_update(C.byref(cfg), _p(gm), _p(gmv), _p(gf), _p(gv), _p(gvt))
    return gv, gvt


def g2p(cfg: Cfg, x, F, gv, gvt, v=None):
    """Sec. 3.4 general transfer to particles.  Returns (x, v, B, F, n_skipped).
    v: the particles' velocities (read by the FLIP transfer only)."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)).copy(); F = _f64(F, (n, d, d)).copy()
    v = np.zeros((n, d)) if v is None else _f64(v, (n, d)).copy()
    B = np.zeros((n, d, d))
    nn = _nodes(cfg)
    bad = _load().or_g2p(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F),
                         _p(_f64(gv, (nn, d))), _p(_f64(gvt, (nn, d))))
    return x, v, B, F, bad


def g2p_lambda0(cfg: Cfg, x, F, gvt):
    """Sec. 5.7 lambda = 0 form of the transfer to particles.  Returns (x, v, B, F, n_skipped)."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)).copy(); F = _f64(F, (n, d, d)).copy()
    v = np.zeros((n, d)); B = np.zeros((n, d, d))
    nn = _nodes(cfg)
    bad = _load().or_g2p_lambda0(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(_f64(gvt, (nn, d))))
    return x, v, B, F, bad


def potential(cfg: Cfg, x, F, vol, dxg) -> float:
    """Phi(x~) = sum_p V_p Psi(F^_p(x~)) with dxg = x~_i - x_i per node (Sec. 3.3)."""
    d = cfg.dim
    n = len(x)
    nn = _nodes(cfg)
    return _load().or_potential(C.byref(cfg), n, _p(_f64(x, (n, d))), _p(_f64(F, (n, d, d))),
                                _p(_f64(np.broadcast_to(vol, (n,)))), _p(_f64(dxg, (nn, d))))


def force_at(cfg: Cfg, x, F, vol, dxg):
    """f_i = -sum_p V_p P(F^_p) (F_p^n)^T grad w_ip with F^_p = (I + sum_i dxg_i grad w^T) F_p^n
    (Sec. 3.3 with F^{n+lambda} = F^_p).  Returns (f, n_skipped)."""
    d = cfg.dim
    n = len(x)
    nn = _nodes(cfg)
    gf = np.zeros((nn, d))
    bad = _load().or_force_at(C.byref(cfg), n, _p(_f64(x, (n, d))), _p(_f64(F, (n, d, d))),
                              _p(_f64(np.broadcast_to(vol, (n,)))), _p(_f64(dxg, (nn, d))), _p(gf))
    return gf, bad


def step_lambda1(cfg: Cfg, x, v, B, F, mass, vol, nsteps: int = 1):
    """nsteps explicit steps of the member lambda = 1 (Sec. 3.3): forces at F^{n+1} from the
    grid velocities before the update, positions moved with them.  Returns (x, v, B, F, skipped)."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)).copy(); v = _f64(v, (n, d)).copy()
    B = _f64(B, (n, d, d)).copy(); F = _f64(F, (n, d, d)).copy()
    mass = _f64(np.broadcast_to(mass, (n,))); vol = _f64(np.broadcast_to(vol, (n,)))
    bad = 0
    for _ in range(nsteps):
        bad += _load().or_step_lambda1(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol))
    return x, v, B, F, bad


def dstress(model: str, F, dF, mu, lam):
    """dP = dP/dF : dF of the fixed-corotated ("fcr") or Neo-Hookean ("nh") stress."""
    F = _f64(F); dF = _f64(dF)
    d = F.shape[0]
    out = np.zeros((d, d))
    fn = _load().or_dstress_nh if model == "nh" else _load().or_dstress_fcr
    fn(d, mu, lam, _p(F), _p(dF), _p(out))
    return out


def force_diff_at(cfg: Cfg, x, F, vol, dxg, du):
    """sum_j (d f_i / d x~_j) du_j at the displacement dxg (Sec. 3.3).  Returns (df, n_skipped)."""
    d = cfg.dim
    n = len(x)
    nn = _nodes(cfg)
    gdf = np.zeros((nn, d))
    bad = _load().or_force_diff_at(C.byref(cfg), n, _p(_f64(x, (n, d))), _p(_f64(F, (n, d, d))),
                                   _p(_f64(np.broadcast_to(vol, (n,)))), _p(_f64(dxg, (nn, d))),
                                   _p(_f64(du, (nn, d))), _p(gdf))
    return gdf, bad


def midpoint_solve(cfg: Cfg, x, F, vol, gm, gv, newton: int = 20, cg: int = 200, tol: float = 1e-13, dv=None):
    """The grid solve of the implicit midpoint rule: dv = v~ - v with
    m_i dv_i = dt f_i(x_i + dt/2 v_i + dt/4 dv_i).  Returns (dv, Newton iterations)."""
    d = cfg.dim
    n = len(x)
    nn = _nodes(cfg)
    dv = np.zeros((nn, d)) if dv is None else _f64(dv, (nn, d)).copy()
    it = _load().or_midpoint_solve(C.byref(cfg), n, _p(_f64(x, (n, d))), _p(_f64(F, (n, d, d))),
                                   _p(_f64(np.broadcast_to(vol, (n,)))), _p(_f64(gm)), _p(_f64(gv, (nn, d))),
                                   newton, cg, tol, _p(dv))
    return dv, it


def step_midpoint(cfg: Cfg, x, v, B, F, mass, vol, newton: int = 20, cg: int = 200, tol: float = 1e-13):
    """One implicit midpoint step (lambda = 1/2, Sec. 4.1-4.2): Newton on the grid velocity
    change, each system by mass-inner-product conjugate gradients (Algorithm 1).
    Returns (x, v, B, F, skipped)."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)).copy(); v = _f64(v, (n, d)).copy()
    B = _f64(B, (n, d, d)).copy(); F = _f64(F, (n, d, d)).copy()
    mass = _f64(np.broadcast_to(mass, (n,))); vol = _f64(np.broadcast_to(vol, (n,)))
    bad = _load().or_step_midpoint(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol),
                                   newton, cg, tol)
    return x, v, B, F, bad


def momentum_particles(cfg: Cfg, x, v, B, mass):
    """Total p and l on particles, l including m_p (B_p)^T : eps (Sec. 5.3)."""
    d = cfg.dim
    n = len(x)
    p = np.zeros(3); l = np.zeros(3)
    _load().or_momentum_particles(C.byref(cfg), n, _p(_f64(x, (n, d))), _p(_f64(v, (n, d))),
                                  _p(_f64(B, (n, d, d))), _p(_f64(np.broadcast_to(mass, (n,)))),
                                  _p(p), _p(l))
    return p, l


def momentum_grid(cfg: Cfg, gmv):
    """Total p and l on the grid, l = sum_i x_i x (m v)_i (Sec. 5.3)."""
    p = np.zeros(3); l = np.zeros(3)
    _load().or_momentum_grid(C.byref(cfg), _p(_f64(gmv, (_nodes(cfg), cfg.dim))), _p(p), _p(l))
    return p, l


def keys(cfg: Cfg, block_edge: int, cell, off) -> np.ndarray:
    """Cell keys from (integer cell, offset in [0,1)) positions."""
    d = cfg.dim
    cell = np.ascontiguousarray(cell, dtype=np.int32).reshape(-1, d)
    off = _f64(off).reshape(-1, d)
    n = len(cell)
    out = np.zeros(n, dtype=np.uint32)
    _load().or_keys(C.byref(cfg), block_edge, n, _p(cell), _p(off), _p(out))
    return out


def stable_sort(k) -> np.ndarray:
    """Permutation of the stable sort of keys (ties by original index)."""
    k = np.ascontiguousarray(k, dtype=np.uint32)
    perm = np.zeros(len(k), dtype=np.int64)
    _load().or_stable_sort(len(k), _p(k), _p(perm))
    return perm


def step(cfg: Cfg, x, v, B, F, mass, vol, nsteps: int = 1, mu=None, lam=None):
    """nsteps whole explicit steps: P2G, grid update, G2P.  Returns (x, v, B, F, skipped).
    mu, lam: per-particle Lame parameters (a material per particle); None = the config's."""
    d = cfg.dim
    n = len(x)
    x = _f64(x, (n, d)).copy(); v = _f64(v, (n, d)).copy()
    B = _f64(B, (n, d, d)).copy(); F = _f64(F, (n, d, d)).copy()
    mass = _f64(np.broadcast_to(mass, (n,))); vol = _f64(np.broadcast_to(vol, (n,)))
    if mu is not None:
        mu = _f64(np.broadcast_to(mu, (n,))); lam = _f64(np.broadcast_to(lam, (n,)))
    bad = 0
    for _ in range(nsteps):
        if mu is None:
            bad += _load().or_step(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol))
        else:
            bad += _load().or_step_mat(C.byref(cfg), n, _p(x), _p(v), _p(B), _p(F), _p(mass), _p(vol),
                                       _p(mu), _p(lam))
    return x, v, B, F, bad
