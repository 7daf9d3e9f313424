"""ctypes wrapper around ``lbm_oracle.c`` -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain single-threaded FP64 C implementation of the method of
Li, Ho, Wu & Zhang (arXiv:1609.09685, Sec. 2): D2Q9 / D3Q19 BGK with Zou-He
pressure boundaries, specular symmetry planes and halfway bounce-back, iterated
to steady state; Darcy permeability from the mass flow rate; Kn =
sqrt(pi/6)(tau - 1/2)/N_x; and the QSGS porous-mask generator.  It shares no
code with the CUDA library.  Arrays are dense numpy arrays with x fastest:
masks ``uint8[nz, ny, nx]`` (``[ny, nx]`` in 2D, 1 = solid) and populations
``float64[nz, ny, nx, Q]`` (unshifted).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

EQ_QUADRATIC = 0
EQ_LINEAR = 1

__all__ = [
    "EQ_QUADRATIC", "EQ_LINEAR", "build", "lattice", "init", "step", "run",
    "equilibrium", "fields", "mean_jx", "permeability", "knudsen", "link_flux",
    "run_to_steady", "splitmix64", "qsgs_hash", "qsgs", "qsgs_grow_once", "percolates",
    "Q_OF", "tau_minus", "pore_d2", "local_knudsen", "step_forced", "run_forced",
    "permeability_forced", "run_forced_to_steady",
]

Q_OF = {2: 9, 3: 19}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 -ffp-contract=off (no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i, d, l, u64, u32 = C.c_int, C.c_double, C.c_long, C.c_uint64, C.c_uint32
            sig = {
                "oc_lattice": (i, [i, P, P, P]),
                "oc_step": (i, [i, i, i, i, P, d, d, d, i, P, P]),
                "oc_run": (i, [i, i, i, i, P, d, d, d, i, P, l]),
                "oc_step_trt": (i, [i, i, i, i, P, d, d, d, d, i, P, P]),
                "oc_run_trt": (i, [i, i, i, i, P, d, d, d, d, i, P, l]),
                "oc_run_to_steady_trt": (i, [i, i, i, i, P, d, d, d, d, i, P, d, l, i, P, P]),
                "oc_init": (i, [i, i, i, i, P, d, d, P]),
                "oc_equilibrium": (i, [i, i, i, i, P, i, P, P, P, P, P]),
                "oc_fields": (i, [i, i, i, i, P, P, P, P, P, P]),
                "oc_mean_jx": (d, [i, i, i, i, P, P]),
                "oc_permeability": (d, [i, i, i, i, P, P, d, d, d]),
                "oc_knudsen": (d, [d, i]),
                "oc_link_flux": (i, [i, i, i, i, P, P, P]),
                "oc_run_to_steady": (i, [i, i, i, i, P, d, d, d, i, P, d, l, i, P, P]),
                "oc_splitmix64": (u64, [u64, u64]),
                "oc_qsgs_hash": (u32, [u64, u32, u64, u32]),
                "oc_qsgs": (i, [i, i, i, u64, d, d, d, P]),
                "oc_qsgs_grow_once": (i, [i, i, i, u64, u32, d, P, P]),
                "oc_percolates": (i, [i, i, i, P]),
                "oc_pore_d2": (i, [i, i, i, P, P]),
                "oc_step_forced": (i, [i, i, i, i, P, d, d, i, P, P]),
                "oc_run_forced": (i, [i, i, i, i, P, d, d, d, i, P, l]),
                "oc_step_forced_trt": (i, [i, i, i, i, P, d, d, d, i, P, P]),
                "oc_permeability_forced": (d, [i, i, i, i, P, P, d, d, d]),
                "oc_local_knudsen": (i, [i, i, i, P, d, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(mask: np.ndarray):
    if mask.ndim == 2:
        return 9, mask.shape[1], mask.shape[0], 1
    if mask.ndim == 3:
        return 19, mask.shape[2], mask.shape[1], mask.shape[0]
    raise ValueError("mask must be [ny, nx] or [nz, ny, nx]")


def _mask(mask):
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.size and m.max() > 1:
        raise ValueError("mask bytes must be 0 (fluid) or 1 (solid)")
    return m


def _fshape(mask):
    q, nx, ny, nz = _dims(mask)
    return mask.shape + (q,)


def lattice(q: int):
    """(c[Q,3] int, w[Q] float64, opp[Q] int) of the oracle's lattice."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    o = np.zeros(q, np.int32)
    if _get().oc_lattice(q, _p(c), _p(w), _p(o)):
        raise ValueError(q)
    return c, w, o


def init(mask, rho_in: float, rho_out: float) -> np.ndarray:
    """Rest equilibrium with rho linear in x from rho_in to rho_out."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    f = np.zeros(_fshape(mask), np.float64)
    if _get().oc_init(q, nx, ny, nz, _p(mask), rho_in, rho_out, _p(f)):
        raise ValueError("bad dimensions")
    return f


def tau_minus(tau: float, lam: float) -> float:
    """TRT antisymmetric relaxation time for the magic parameter
    Lambda = (tau - 1/2)(tau_minus - 1/2)."""
    return 0.5 + lam / (tau - 0.5)


def step(mask, f, tau, rho_in, rho_out, eq=EQ_QUADRATIC, tau_m=None) -> np.ndarray:
    """One stream + boundary + collide step; returns the new post-collision state.
    tau_m: TRT antisymmetric relaxation time (None = BGK)."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    fin = np.ascontiguousarray(f, np.float64)
    out = np.zeros_like(fin)
    if tau_m is None:
        rc = _get().oc_step(q, nx, ny, nz, _p(mask), tau, rho_in, rho_out, eq, _p(fin), _p(out))
    else:
        rc = _get().oc_step_trt(q, nx, ny, nz, _p(mask), tau, tau_m, rho_in, rho_out, eq, _p(fin), _p(out))
    if rc:
        raise ValueError("bad arguments")
    return out


def run(mask, f, tau, rho_in, rho_out, nsteps, eq=EQ_QUADRATIC, tau_m=None) -> np.ndarray:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    g = np.array(f, np.float64, copy=True, order="C")
    if _get().oc_run_trt(q, nx, ny, nz, _p(mask), tau, 0.0 if tau_m is None else tau_m, rho_in, rho_out,
                         eq, _p(g), int(nsteps)):
        raise ValueError("bad arguments")
    return g


def equilibrium(mask, rho, ux, uy, uz=None, eq=EQ_QUADRATIC) -> np.ndarray:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (rho, ux, uy)]
    uzp = None if uz is None else np.ascontiguousarray(uz, np.float64)
    f = np.zeros(_fshape(mask), np.float64)
    _get().oc_equilibrium(q, nx, ny, nz, _p(mask), eq, *[_p(a) for a in arrs],
                          None if uzp is None else _p(uzp), _p(f))
    return f


def fields(mask, f):
    """(rho, ux, uy[, uz]) dense, zero on solids."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    f = np.ascontiguousarray(f, np.float64)
    out = [np.zeros(mask.shape, np.float64) for _ in range(4 if q == 19 else 3)]
    _get().oc_fields(q, nx, ny, nz, _p(mask), _p(f), *[_p(a) for a in out[:3]],
                     _p(out[3]) if q == 19 else None)
    return tuple(out)


def mean_jx(mask, f) -> float:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    return _get().oc_mean_jx(q, nx, ny, nz, _p(mask), _p(np.ascontiguousarray(f, np.float64)))


def permeability(mask, f, tau, rho_in, rho_out) -> float:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    return _get().oc_permeability(q, nx, ny, nz, _p(mask),
                                  _p(np.ascontiguousarray(f, np.float64)), tau, rho_in, rho_out)


def knudsen(tau: float, nx: int) -> float:
    return _get().oc_knudsen(tau, nx)


def link_flux(mask, f) -> np.ndarray:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    out = np.zeros(nx - 1, np.float64)
    _get().oc_link_flux(q, nx, ny, nz, _p(mask), _p(np.ascontiguousarray(f, np.float64)), _p(out))
    return out


def run_to_steady(mask, f, tau, rho_in, rho_out, tol, max_steps, interval=100,
                  eq=EQ_QUADRATIC, tau_m=None):
    """Iterate in place-copy; returns (f, status, steps, residual).

    status 0 = converged (r < tol), 1 = max_steps reached."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    g = np.array(f, np.float64, copy=True, order="C")
    steps = C.c_long(0)
    res = C.c_double(0.0)
    rc = _get().oc_run_to_steady_trt(q, nx, ny, nz, _p(mask), tau, 0.0 if tau_m is None else tau_m, rho_in,
                                     rho_out, eq, _p(g), tol, int(max_steps), int(interval), C.byref(steps),
                                     C.byref(res))
    if rc < 0:
        raise RuntimeError(f"oracle run_to_steady failed ({rc})")
    return g, rc, steps.value, res.value


def splitmix64(seed: int, n: int) -> int:
    """The n-th (n >= 1) output of splitmix64 started from seed."""
    return int(_get().oc_splitmix64(seed & (2**64 - 1), n))


def qsgs_hash(seed: int, t: int, cell: int, d: int) -> int:
    return int(_get().oc_qsgs_hash(seed & (2**64 - 1), t, cell, d))


def qsgs(shape, seed: int, core_p: float, porosity: float, d_face: float = 0.2):
    """QSGS mask of shape (ny, nx) or (nz, ny, nx); returns (mask, iterations)."""
    if len(shape) == 2:
        nz, (ny, nx) = 1, shape
    else:
        nz, ny, nx = shape
    m = np.zeros((nz, ny, nx), np.uint8)
    it = _get().oc_qsgs(nx, ny, nz, seed & (2**64 - 1), core_p, porosity, d_face, _p(m))
    if it < 0:
        raise RuntimeError(f"oracle qsgs failed ({it})")
    return (m[0] if len(shape) == 2 else m), it


def qsgs_grow_once(start, seed: int, t: int, d_face: float = 0.2) -> np.ndarray:
    """Candidate cells (uint8) of growth iteration t >= 1 from mask `start`."""
    st = _mask(start)
    sh = st.shape if st.ndim == 3 else (1,) + st.shape
    out = np.zeros(st.shape, np.uint8)
    rc = _get().oc_qsgs_grow_once(sh[2], sh[1], sh[0], seed & (2**64 - 1), t, d_face,
                                  _p(st), _p(out))
    if rc < 0:
        raise RuntimeError(rc)
    return out


def percolates(mask) -> bool:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    return bool(_get().oc_percolates(nx, ny, nz, _p(mask)))


def pore_d2(mask) -> np.ndarray:
    """Squared distance (nodes) from each node to the nearest solid node; 0 on
    solids, 2**32 - 1 where the domain has no solid."""
    mask = _mask(mask)
    _, nx, ny, nz = _dims(mask)
    out = np.zeros(mask.shape, np.uint32)
    if _get().oc_pore_d2(nx, ny, nz, _p(mask), _p(out)):
        raise ValueError("bad arguments")
    return out


def local_knudsen(mask, tau):
    """(h, Kn): local pore size 2 D - 1 and local Knudsen number
    sqrt(pi/6)(tau - 1/2)/h on fluid nodes, 0 on solids."""
    mask = _mask(mask)
    _, nx, ny, nz = _dims(mask)
    h = np.zeros(mask.shape, np.float64)
    kn = np.zeros(mask.shape, np.float64)
    if _get().oc_local_knudsen(nx, ny, nz, _p(mask), tau, _p(h), _p(kn)):
        raise ValueError("bad arguments")
    return h, kn


def step_forced(mask, f, tau, g, eq=EQ_QUADRATIC, tau_m=None) -> np.ndarray:
    """One step of force-driven flow with every face periodic (body
    acceleration g along +x, Guo forcing); tau_m: TRT (None = BGK)."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    fin = np.ascontiguousarray(f, np.float64)
    out = np.zeros_like(fin)
    if tau_m is None:
        rc = _get().oc_step_forced(q, nx, ny, nz, _p(mask), tau, g, eq, _p(fin), _p(out))
    else:
        rc = _get().oc_step_forced_trt(q, nx, ny, nz, _p(mask), tau, tau_m, g, eq, _p(fin), _p(out))
    if rc:
        raise ValueError("bad arguments")
    return out


def run_forced(mask, f, tau, g, nsteps, eq=EQ_QUADRATIC, tau_m=None) -> np.ndarray:
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    h = np.array(f, np.float64, copy=True, order="C")
    if _get().oc_run_forced(q, nx, ny, nz, _p(mask), tau, 0.0 if tau_m is None else tau_m, g, eq, _p(h),
                            int(nsteps)):
        raise ValueError("bad arguments")
    return h


def permeability_forced(mask, f, tau, g, rho0=1.0) -> float:
    """Eq. (2): k = nu <u>/g over all grid nodes."""
    mask = _mask(mask)
    q, nx, ny, nz = _dims(mask)
    return _get().oc_permeability_forced(q, nx, ny, nz, _p(mask), _p(np.ascontiguousarray(f, np.float64)),
                                         tau, g, rho0)


def run_forced_to_steady(mask, f, tau, g, tol, max_steps, interval=100, eq=EQ_QUADRATIC, tau_m=None):
    """Steps in intervals until the relative velocity change over an interval
    is below tol; returns (f, status, steps, residual), status 0 = converged."""
    mask = _mask(mask)
    h = np.array(f, np.float64, copy=True, order="C")
    fl = ~mask.astype(bool)
    prev = np.stack(fields(mask, h)[1:], axis=-1)[fl]
    steps, r = 0, np.inf
    while steps < max_steps:
        h = run_forced(mask, h, tau, g, interval, eq, tau_m)
        steps += interval
        cur = np.stack(fields(mask, h)[1:], axis=-1)[fl]
        den = np.sqrt((cur ** 2).sum())
        r = np.sqrt(((cur - prev) ** 2).sum()) / den if den > 0 else np.inf
        prev = cur
        if r < tol:
            return h, 0, steps, r
    return h, 1, steps, r
