"""Thin ctypes binding of ``include/lbm.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of the method: numpy arrays are passed as host pointers, results
are copied back, and a non-OK status raises :class:`LBMError`.  The CUDA
library must have been built (``python -m paper_1609_09685_gb300.build``);
importing the binding without it fails loudly.  PyTorch supplies only the CUDA
stream (``torch.cuda.current_stream()``) when the caller asks for it.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_NOT_CONVERGED = 1
LBM_STALLED = 2
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_DIVERGED = -4
LBM_TIMEOUT = -5
LBM_ERR_IO = -6
LBM_ERR_INTERNAL = -7
LBM_CANCELLED = -8
LBM_EQ_QUADRATIC = 0
LBM_EQ_LINEAR = 1
LBM_COLL_BGK = 0
LBM_COLL_TRT = 1
NUM_OBS = 8

# informational statuses that do not raise
_SOFT = (LBM_OK, LBM_NOT_CONVERGED, LBM_STALLED)


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class lbm_options(C.Structure):
    _fields_ = [
        ("struct_size", C.c_int32),
        ("equilibrium", C.c_int32),
        ("check_interval", C.c_int32),
        ("stall_checks", C.c_int32),
        ("stall_floor", C.c_double),
        ("rho_out", C.c_double),
        ("stream", C.c_void_p),
        ("block_threads", C.c_int32),
        ("use_graphs", C.c_int32),
        ("cancel_flag", C.c_void_p),
        ("strip_rows", C.c_int32),
        ("k_tol", C.c_double),
        ("in_place_pairs", C.c_int32),
        ("collision", C.c_int32),
        ("trt_lambda", C.c_double),
        ("tile_rows", C.c_int32),
        ("gather_batch", C.c_int32),
        ("autotune", C.c_int32),
        ("tune_cache", C.c_char_p),
        ("alloc_fn", C.c_void_p),
        ("free_fn", C.c_void_p),
        ("alloc_ctx", C.c_void_p),
        ("band_rows", C.c_int32),
        ("pair_block_mb", C.c_int32),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


def torch_allocator(fail_after: Optional[int] = None, log: Optional[list] = None):
    """(alloc_fn, free_fn) callbacks that lend PyTorch's CUDA caching allocator
    to a solver (pass them to make_options).  fail_after: the allocation with
    that index (0-based) and every later one return NULL -- an injected
    out-of-memory for tests.  log: receives ("alloc", ptr, bytes) and
    ("free", ptr) events."""
    import torch
    count = [0]

    def _alloc(ctx, nbytes, stream):
        i = count[0]
        count[0] += 1
        if fail_after is not None and i >= fail_after:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        if log is not None:
            log.append(("alloc", int(p), int(nbytes)))
        return int(p)

    def _free(ctx, ptr, stream):
        if log is not None:
            log.append(("free", int(ptr)))
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free)


class lbm_launch(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("strip_rows", C.c_int32), ("gather_batch", C.c_int32),
                ("tile_rows", C.c_int32), ("band_rows", C.c_int32), ("pair_block_mb", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_tune_result(C.Structure):
    _fields_ = [("chosen", lbm_launch), ("us_per_step", C.c_double), ("defaults", lbm_launch),
                ("us_per_step_default", C.c_double), ("candidates", C.c_int32), ("from_cache", C.c_int32)]


class lbm_domain_desc(C.Structure):
    _fields_ = [
        ("mask", C.c_void_p),
        ("nx", C.c_int32),
        ("ny", C.c_int32),
        ("nz", C.c_int32),
        ("tau", C.c_double),
        ("drho", C.c_double),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load the CUDA library (raises if it has not been built).  A path loads
    that build instead (for instance the checked one) and makes it the
    library every function of this module calls, until `unload()`."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(
            f"CUDA library {p} is missing: build it with `python -m paper_1609_09685_gb300.build`")
    lib = C.CDLL(p)
    P, i32, i64, d, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
    sigs = {
        "lbm_version": (C.c_char_p, []),
        "lbm_status_string": (C.c_char_p, [i32]),
        "lbm_last_error": (C.c_char_p, [P]),
        "lbm_options_default": (None, [P]),
        "lbm_qsgs": (i32, [u64, i32, i32, i32, d, d, d, P, P, P]),
        "lbm_qsgs_noalloc": (i32, [u64, i32, i32, i32, d, d, d, P, P, P]),
        "lbm_batch_create": (i32, [i32, P, P, P]),
        "lbm_batch_create_forced": (i32, [i32, P, P, P, P]),
        "lbm_create_domain": (i32, [P, i32, i32, d, d, P, P]),
        "lbm_create_domain_3d": (i32, [P, i32, i32, i32, d, d, P, P]),
        "lbm_destroy": (None, [P]),
        "lbm_info": (i32, [P, P, P, P]),
        "lbm_domain_fluid_nodes": (i32, [P, i32, P]),
        "lbm_step": (i32, [P, i64]),
        "lbm_step_observe": (i32, [P, i64, P]),
        "lbm_profile_steps": (i32, [P, i64, P, P]),
        "lbm_local_knudsen": (i32, [P, i32, P, P, P]),
        "lbm_run_to_steady": (i32, [P, d, i64, P, P, P]),
        "lbm_permeability": (i32, [P, P, P]),
        "lbm_batch_run_to_steady": (i32, [P, d, i64, P]),
        "lbm_batch_permeability": (i32, [P, P]),
        "lbm_batch_destroy": (None, [P]),
        "lbm_lattice": (i32, [i32, P, P, P, P, P]),
        "lbm_slab_create": (i32, [P, i32, i32, i32, d, d, i32, i32, i32, P, P]),
        "lbm_slab_halo_floats": (i32, [P, i32, i32, P]),
        "lbm_slab_export": (i32, [P, i32, P]),
        "lbm_slab_import": (i32, [P, i32, P]),
        "lbm_slab_observables": (i32, [P, P, P, P, P]),
        "lbm_build_checked": (i32, [P]),
        "lbm_debug_corrupt_window": (i32, [P, C.c_uint32, C.c_uint32]),
        "lbm_get_launch": (i32, [P, P]),
        "lbm_set_launch": (i32, [P, P]),
        "lbm_time_steps": (i32, [P, i32, P]),
        "lbm_autotune": (i32, [P, C.c_char_p, i32, P]),
        "lbm_tune_key": (i32, [P, P, C.c_size_t]),
        "lbm_tune_key_for": (i32, [C.c_char_p, i32, i64, i32, i32, P, C.c_size_t]),
        "lbm_tune_cache_get": (i32, [C.c_char_p, C.c_char_p, P, P, P]),
        "lbm_tune_cache_put": (i32, [C.c_char_p, C.c_char_p, P, d]),
        "lbm_get_fields": (i32, [P, i32, P, P, P, P]),
        "lbm_get_populations": (i32, [P, i32, P]),
        "lbm_set_populations": (i32, [P, i32, P]),
        "lbm_set_fields": (i32, [P, i32, P, P, P, P, i32]),
        "lbm_get_step": (i32, [P, P]),
        "lbm_get_history": (i32, [P, i32, P, P, P, P, i32, P]),
        "lbm_nn_set_conv_impl": (i32, [i32]),
        "lbm_nn_get_conv_impl": (i32, []),
        "lbm_nn_sync_status": (i32, [P]),
        "lbm_nn_conv_fwd": (i32, [P, i32, i32, i32, i32, P, P, i32, i32, i32, P, P, P]),
        "lbm_nn_conv_bwd_data": (i32, [P, i32, i32, i32, i32, P, i32, i32, P, P, P]),
        "lbm_nn_conv_bwd_weight": (i32, [P, P, i32, i32, i32, i32, i32, i32, P, P, i32, P, C.c_size_t, P]),
        "lbm_nn_relu_bwd": (i32, [P, P, P, C.c_size_t, P]),
        "lbm_nn_pool2_fwd": (i32, [P, i32, i32, i32, i32, P, P]),
        "lbm_nn_pool2_bwd": (i32, [P, i32, i32, i32, i32, P, P]),
        "lbm_nn_up2_fwd": (i32, [P, i32, i32, i32, i32, P, P]),
        "lbm_nn_up2_bwd": (i32, [P, i32, i32, i32, i32, P, P]),
        "lbm_nn_copy_channels": (i32, [P, i32, i32, P, i32, i32, i32, C.c_size_t, P]),
        "lbm_nn_mse": (i32, [P, i32, P, P, C.c_size_t, i32, P, C.c_float, P, P, P, P]),
        "lbm_nn_adamw": (i32, [P, P, P, P, C.c_size_t, C.c_float, C.c_float, C.c_float, C.c_float,
                               C.c_float, i32, P, P]),
        "lbm_nn_f32_to_bf16": (i32, [P, P, C.c_size_t, P]),
        "lbm_nn_add": (i32, [P, P, P, C.c_size_t, P]),
        "lbm_nn_make_input": (i32, [P, i32, i32, C.c_float, P, P]),
        "lbm_nn_targets": (i32, [P, i32, P]),
        "lbm_warm_start": (i32, [P, i32, P, i32]),
        "lbm_save": (i32, [P, C.c_char_p]),
        "lbm_load": (i32, [C.c_char_p, P, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def unload() -> None:
    """Forget the loaded library handle (the next call loads the default build)."""
    global _lib
    _lib = None


def _check(st: int, handle=None, soft=_SOFT) -> int:
    if st in soft:
        return st
    msg = load().lbm_last_error(handle).decode(errors="replace")
    raise LBMError(st, msg or load().lbm_status_string(st).decode())


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def current_stream() -> Optional[int]:
    """torch's current CUDA stream handle, or None."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return None


def make_options(equilibrium=LBM_EQ_QUADRATIC, check_interval=100, stall_checks=200,
                 stall_floor=1e-5, rho_out=1.0, stream=None, block_threads=0,
                 use_graphs=True, cancel_flag=None, strip_rows=0, k_tol=1e-5,
                 in_place_pairs=True, collision=0, trt_lambda=3.0 / 16.0, tile_rows=0, gather_batch=0,
                 autotune=False, tune_cache=None, allocator=None, band_rows=0, pair_block_mb=0) -> lbm_options:
    o = lbm_options()
    load().lbm_options_default(C.byref(o))
    o.equilibrium = equilibrium
    o.check_interval = check_interval
    o.stall_checks = stall_checks
    o.stall_floor = stall_floor
    o.rho_out = rho_out
    o.stream = stream
    o.block_threads = block_threads
    o.use_graphs = 1 if use_graphs else 0
    o.cancel_flag = cancel_flag
    o.strip_rows = strip_rows
    o.k_tol = k_tol
    o.in_place_pairs = 1 if in_place_pairs else 0
    o.collision = collision
    o.trt_lambda = trt_lambda
    o.tile_rows = tile_rows
    o.gather_batch = gather_batch
    o.band_rows = band_rows
    o.pair_block_mb = pair_block_mb
    o.autotune = 1 if autotune else 0
    o.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
    if allocator is not None:  # (alloc_fn, free_fn) callbacks, kept alive by the options object
        o._allocator = allocator
        o.alloc_fn = C.cast(allocator[0], C.c_void_p)
        o.free_fn = C.cast(allocator[1], C.c_void_p)
    return o


def _mask(m) -> np.ndarray:
    a = np.ascontiguousarray(m, dtype=np.uint8)
    if a.ndim not in (2, 3):
        raise ValueError("mask must be [ny, nx] or [nz, ny, nx]")
    return a


def lbm_version() -> str:
    return load().lbm_version().decode()


def lbm_qsgs(seed: int, shape: Sequence[int], core_p: float, porosity: float,
             d_face: float = 0.2, stream=None):
    """QSGS mask (uint8, shape (ny, nx) or (nz, ny, nx)) and iteration count."""
    if len(shape) == 2:
        nz, (ny, nx) = 1, shape
    else:
        nz, ny, nx = shape
    out = np.zeros((nz, ny, nx), np.uint8)
    it = C.c_int32(0)
    _check(load().lbm_qsgs(seed & (2**64 - 1), nx, ny, nz, core_p, porosity, d_face, stream,
                           _ptr(out), C.byref(it)))
    return (out[0] if len(shape) == 2 else out), it.value


def lbm_qsgs_noalloc(seed: int, shape: Sequence[int], core_p: float, porosity: float,
                     mask_dev_ptr: int, d_face: float = 0.2, stream=None) -> int:
    """QSGS mask written to a caller-owned device buffer (device pointer
    mask_dev_ptr, nx*ny*nz bytes) with no allocation; returns the iteration count."""
    if len(shape) == 2:
        nz, (ny, nx) = 1, shape
    else:
        nz, ny, nx = shape
    it = C.c_int32(0)
    _check(load().lbm_qsgs_noalloc(seed & (2**64 - 1), nx, ny, nz, core_p, porosity, d_face, stream,
                                   C.c_void_p(int(mask_dev_ptr)), C.byref(it)))
    return it.value


class Solver:
    """Owner of an ``lbm_handle`` (a batch of one or more domains)."""

    def __init__(self, handle: C.c_void_p, masks, taus, drhos, options: lbm_options):
        self._h = handle
        self.masks = masks
        self.taus = list(taus)
        self.drhos = list(drhos)
        self.options = options
        n, q, nf = C.c_int32(), C.c_int32(), C.c_int64()
        _check(load().lbm_info(self._h, C.byref(n), C.byref(q), C.byref(nf)), self._h)
        self.n_domains, self.q, self.fluid_nodes = n.value, q.value, nf.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().lbm_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def lbm_batch_create(masks: Sequence[np.ndarray], taus: Sequence[float], drhos: Sequence[float],
                     options: Optional[lbm_options] = None) -> Solver:
    masks = [_mask(m) for m in masks]
    n = len(masks)
    descs = (lbm_domain_desc * n)()
    for k, m in enumerate(masks):
        if m.ndim == 2:
            nz, (ny, nx) = 1, m.shape
        else:
            nz, ny, nx = m.shape
        descs[k] = lbm_domain_desc(m.ctypes.data, nx, ny, nz, float(taus[k]), float(drhos[k]))
    o = options or make_options()
    h = C.c_void_p()
    _check(load().lbm_batch_create(n, descs, C.byref(o), C.byref(h)))
    return Solver(h, masks, taus, drhos, o)


def lbm_batch_create_forced(masks: Sequence[np.ndarray], taus: Sequence[float], g: Sequence[float],
                            options: Optional[lbm_options] = None) -> Solver:
    """Force-driven domains with every face periodic (body acceleration g[d]
    along +x); lbm_permeability gives Eq. 2's k = nu <u>/g."""
    masks = [_mask(m) for m in masks]
    n = len(masks)
    descs = (lbm_domain_desc * n)()
    for d, m in enumerate(masks):
        nz, ny, nx = (1,) + m.shape if m.ndim == 2 else m.shape
        descs[d] = lbm_domain_desc(m.ctypes.data, nx, ny, nz, float(taus[d]), 0.0)
    gg = np.ascontiguousarray(g, np.float64)
    o = options if options is not None else make_options()
    h = C.c_void_p()
    _check(load().lbm_batch_create_forced(n, descs, _ptr(gg), C.byref(o), C.byref(h)))
    return Solver(h, masks, taus, [0.0] * n, o)


def lbm_create_domain(mask, tau: float, drho: float, options: Optional[lbm_options] = None) -> Solver:
    m = _mask(mask)
    if m.ndim != 2:
        raise ValueError("lbm_create_domain takes a 2D mask; use lbm_create_domain_3d")
    o = options or make_options()
    h = C.c_void_p()
    _check(load().lbm_create_domain(_ptr(m), m.shape[1], m.shape[0], tau, drho, C.byref(o),
                                    C.byref(h)))
    return Solver(h, [m], [tau], [drho], o)


def lbm_create_domain_3d(mask, tau: float, drho: float,
                         options: Optional[lbm_options] = None) -> Solver:
    m = _mask(mask)
    if m.ndim != 3:
        raise ValueError("lbm_create_domain_3d takes a [nz, ny, nx] mask")
    o = options or make_options()
    h = C.c_void_p()
    nz, ny, nx = m.shape
    _check(load().lbm_create_domain_3d(_ptr(m), nx, ny, nz, tau, drho, C.byref(o), C.byref(h)))
    return Solver(h, [m], [tau], [drho], o)


def lbm_domain_fluid_nodes(s: Solver, d: int) -> int:
    v = C.c_int64()
    _check(load().lbm_domain_fluid_nodes(s.handle, d, C.byref(v)), s.handle)
    return v.value


def lbm_step(s: Solver, nsteps: int) -> None:
    _check(load().lbm_step(s.handle, int(nsteps)), s.handle)


def lbm_step_observe(s: Solver, nsteps: int) -> np.ndarray:
    out = np.zeros((s.n_domains, NUM_OBS), np.float64)
    _check(load().lbm_step_observe(s.handle, int(nsteps), _ptr(out)), s.handle)
    return out


def lbm_local_knudsen(s: Solver, d: int):
    """(d2, h, kn) of domain d in the mask's shape: squared distance to the
    nearest solid node, local pore size 2 D - 1 and local Knudsen number."""
    shape = s.masks[d].shape
    n_nodes = int(np.prod(shape))
    d2 = np.zeros(n_nodes, np.uint32)
    h = np.zeros(n_nodes, np.float64)
    kn = np.zeros(n_nodes, np.float64)
    _check(load().lbm_local_knudsen(s.handle, int(d), _ptr(d2), _ptr(h), _ptr(kn)), s.handle)
    return d2.reshape(shape), h.reshape(shape), kn.reshape(shape)


def lbm_status_string(status: int) -> str:
    return load().lbm_status_string(int(status)).decode()


def lbm_last_error(s: Optional["Solver"] = None) -> str:
    """Detail of the last failure on this handle (None: this thread's last
    failure outside a handle)."""
    return load().lbm_last_error(s.handle if s is not None else None).decode(errors="replace")


def lbm_options_default() -> lbm_options:
    o = lbm_options()
    load().lbm_options_default(C.byref(o))
    return o


def lbm_info(s: "Solver"):
    """(number of domains, Q, total fluid nodes)."""
    n, q, nf = C.c_int32(), C.c_int32(), C.c_int64()
    _check(load().lbm_info(s.handle, C.byref(n), C.byref(q), C.byref(nf)), s.handle)
    return n.value, q.value, nf.value


def lbm_destroy(s: "Solver") -> None:
    s.close()


KERNEL_KINDS = ("gather", "local", "pull", "pull_observe", "pair_fused")


def lbm_profile_steps(s: Solver, nsteps: int) -> dict:
    """nsteps plain steps with CUDA events around every kernel; returns
    {kind: (total device microseconds, launches)}."""
    t = np.zeros(len(KERNEL_KINDS), np.float64)
    c = np.zeros(len(KERNEL_KINDS), np.int64)
    _check(load().lbm_profile_steps(s.handle, int(nsteps), _ptr(t), _ptr(c)), s.handle)
    return {k: (float(t[i]), int(c[i])) for i, k in enumerate(KERNEL_KINDS)}


def lbm_run_to_steady(s: Solver, tol: float, max_steps: int):
    """Returns (overall status, per-domain status, steps, residual)."""
    n = s.n_domains
    st = np.zeros(n, np.int32)
    steps = np.zeros(n, np.int64)
    res = np.zeros(n, np.float64)
    rc = _check(load().lbm_run_to_steady(s.handle, tol, int(max_steps), _ptr(st), _ptr(steps),
                                         _ptr(res)), s.handle)
    return rc, st, steps, res


def lbm_permeability(s: Solver):
    """(k[n], kn[n]) from the last observation."""
    k = np.zeros(s.n_domains, np.float64)
    kn = np.zeros(s.n_domains, np.float64)
    _check(load().lbm_permeability(s.handle, _ptr(k), _ptr(kn)), s.handle)
    return k, kn


def lbm_batch_run_to_steady(s: Solver, tol: float, max_steps: int):
    """Returns (overall status, per-domain status)."""
    st = np.zeros(s.n_domains, np.int32)
    rc = _check(load().lbm_batch_run_to_steady(s.handle, tol, int(max_steps), _ptr(st)), s.handle)
    return rc, st


def lbm_batch_permeability(s: Solver) -> np.ndarray:
    """k[n] from the last observation."""
    k = np.zeros(s.n_domains, np.float64)
    _check(load().lbm_batch_permeability(s.handle, _ptr(k)), s.handle)
    return k


def lbm_batch_destroy(s: Solver) -> None:
    """Frees the batch through lbm_batch_destroy; the Solver is closed after."""
    if s._h:
        load().lbm_batch_destroy(s._h)
        s._h = None


def lbm_lattice(q: int):
    """(c[q, 3], w[q], opp[q], flip_y[q], flip_z[q]): the kernels' lattice tables."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    o = np.zeros(q, np.int32)
    fy = np.zeros(q, np.int32)
    fz = np.zeros(q, np.int32)
    _check(load().lbm_lattice(int(q), _ptr(c), _ptr(w), _ptr(o), _ptr(fy), _ptr(fz)))
    return c, w, o, fy, fz


def lbm_slab_create(mask, tau: float, drho: float, x_offset: int, nx_global: int, ghosts: int,
                    options: Optional[lbm_options] = None) -> Solver:
    """One x-slab (ghost columns included in `mask`) of a domain of nx_global columns."""
    m = _mask(mask)
    o = options or make_options()
    h = C.c_void_p()
    nz, ny, nx = (1,) + m.shape if m.ndim == 2 else m.shape
    _check(load().lbm_slab_create(_ptr(m), nx, ny, nz, tau, drho, int(x_offset), int(nx_global), int(ghosts),
                                  C.byref(o), C.byref(h)))
    return Solver(h, [m], [tau], [drho], o)


def lbm_slab_halo_floats(s: Solver, side: int, incoming: bool = False) -> int:
    n = C.c_int64()
    _check(load().lbm_slab_halo_floats(s.handle, int(side), 1 if incoming else 0, C.byref(n)), s.handle)
    return n.value


def lbm_slab_export(s: Solver, side: int, buf) -> None:
    """Pack the real column next to cut `side` into the device buffer `buf`
    (a pointer, or an object with data_ptr())."""
    _check(load().lbm_slab_export(s.handle, int(side), _dp(buf)), s.handle)


def lbm_slab_import(s: Solver, side: int, buf) -> None:
    _check(load().lbm_slab_import(s.handle, int(side), _dp(buf)), s.handle)


def lbm_slab_observables(s: Solver, obs_sum) -> tuple:
    """(k, Kn, residual) of the whole domain from observables summed over its slabs."""
    o = np.ascontiguousarray(obs_sum, np.float64).reshape(-1)
    if o.size < NUM_OBS:
        raise ValueError("need the 8 observables")
    k, kn, r = C.c_double(), C.c_double(), C.c_double()
    _check(load().lbm_slab_observables(s.handle, _ptr(o), C.byref(k), C.byref(kn), C.byref(r)), s.handle)
    return k.value, kn.value, r.value


def lbm_build_checked() -> bool:
    c = C.c_int32()
    _check(load().lbm_build_checked(C.byref(c)))
    return bool(c.value)


def lbm_debug_corrupt_window(s: Solver, seg: int, value: int) -> None:
    _check(load().lbm_debug_corrupt_window(s.handle, int(seg), int(value)), s.handle)


def lbm_get_launch(s: Solver) -> dict:
    c = lbm_launch()
    _check(load().lbm_get_launch(s.handle, C.byref(c)), s.handle)
    return c.as_dict()


def lbm_set_launch(s: Solver, block_threads: int, strip_rows: int, gather_batch: int, tile_rows: int = 0,
                   band_rows: int = 0, pair_block_mb: int = 0) -> None:
    c = lbm_launch(block_threads, strip_rows, gather_batch, tile_rows, band_rows, pair_block_mb)
    _check(load().lbm_set_launch(s.handle, C.byref(c)), s.handle)


def lbm_time_steps(s: Solver, nsteps: int = 20) -> float:
    """Device microseconds per plain step (state saved and restored)."""
    us = C.c_double()
    _check(load().lbm_time_steps(s.handle, int(nsteps), C.byref(us)), s.handle)
    return us.value


def lbm_autotune(s: Solver, cache_path: Optional[str] = None, nsteps: int = 0) -> dict:
    r = lbm_tune_result()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load().lbm_autotune(s.handle, path, int(nsteps), C.byref(r)), s.handle)
    return {"chosen": r.chosen.as_dict(), "us_per_step": r.us_per_step, "defaults": r.defaults.as_dict(),
            "us_per_step_default": r.us_per_step_default, "candidates": r.candidates,
            "from_cache": bool(r.from_cache)}


def lbm_tune_key(s: Solver) -> str:
    buf = C.create_string_buffer(512)
    _check(load().lbm_tune_key(s.handle, buf, 512), s.handle)
    return buf.value.decode()


def lbm_tune_key_for(device_name: str, q: int, fluid_nodes: int, eq: int = 0, collision: int = 0) -> str:
    buf = C.create_string_buffer(512)
    _check(load().lbm_tune_key_for(device_name.encode(), q, int(fluid_nodes), eq, collision, buf, 512))
    return buf.value.decode()


def lbm_tune_cache_get(path: str, key: str):
    """(launch dict, us_per_step) or None."""
    c = lbm_launch()
    us = C.c_double()
    found = C.c_int32()
    _check(load().lbm_tune_cache_get(os.fsencode(path), key.encode(), C.byref(c), C.byref(us), C.byref(found)))
    return (c.as_dict(), us.value) if found.value else None


def lbm_tune_cache_put(path: str, key: str, cfg: dict, us_per_step: float) -> None:
    c = lbm_launch(cfg["block_threads"], cfg["strip_rows"], cfg["gather_batch"], cfg["tile_rows"],
                   cfg.get("band_rows", 0), cfg.get("pair_block_mb", 0))
    _check(load().lbm_tune_cache_put(os.fsencode(path), key.encode(), C.byref(c), float(us_per_step)))


def _shape(s: Solver, d: int):
    return s.masks[d].shape


def lbm_get_fields(s: Solver, d: int = 0):
    shp = _shape(s, d)
    arrs = [np.zeros(shp, np.float64) for _ in range(4)]
    _check(load().lbm_get_fields(s.handle, d, *[_ptr(a) for a in arrs]), s.handle)
    return tuple(arrs[:3] if s.q == 9 else arrs)


def lbm_get_populations(s: Solver, d: int = 0) -> np.ndarray:
    f = np.zeros(_shape(s, d) + (s.q,), np.float64)
    _check(load().lbm_get_populations(s.handle, d, _ptr(f)), s.handle)
    return f


def lbm_set_populations(s: Solver, d: int, f: np.ndarray) -> None:
    a = np.ascontiguousarray(f, np.float64)
    if a.shape != _shape(s, d) + (s.q,):
        raise ValueError(f"expected shape {_shape(s, d) + (s.q,)}")
    _check(load().lbm_set_populations(s.handle, d, _ptr(a)), s.handle)


def lbm_set_fields(s: Solver, d: int, drho, ux, uy, uz=None, on_device: bool = False) -> None:
    """Warm start from dense float32 fields (numpy arrays, or device pointers /
    torch CUDA tensors with on_device=True)."""
    if on_device:
        ptrs = [C.c_void_p(int(a.data_ptr()) if hasattr(a, "data_ptr") else int(a)) if a is not None
                else None for a in (drho, ux, uy, uz)]
        _check(load().lbm_set_fields(s.handle, d, *ptrs, 1), s.handle)
        return
    arrs = [None if a is None else np.ascontiguousarray(a, np.float32) for a in (drho, ux, uy, uz)]
    for a in arrs:
        if a is not None and a.shape != _shape(s, d):
            raise ValueError("field shape mismatch")
    _check(load().lbm_set_fields(s.handle, d, *[None if a is None else _ptr(a) for a in arrs], 0),
           s.handle)


def lbm_get_history(s: Solver, d: int = 0):
    """(steps, k, residual, seconds) per check interval of the last run_to_steady."""
    cnt = C.c_int32(0)
    _check(load().lbm_get_history(s.handle, d, None, None, None, None, 0, C.byref(cnt)), s.handle)
    n = cnt.value
    st = np.zeros(n, np.int64)
    k = np.zeros(n, np.float64)
    r = np.zeros(n, np.float64)
    t = np.zeros(n, np.float64)
    _check(load().lbm_get_history(s.handle, d, _ptr(st), _ptr(k), _ptr(r), _ptr(t), n, C.byref(cnt)),
           s.handle)
    return st, k, r, t


# ---------------------------------------------------------------------------
# warm-start network kernels: device pointers (ints, or objects with
# data_ptr(), e.g. torch CUDA tensors) in, nothing computed here
# ---------------------------------------------------------------------------
def _dp(t):
    if t is None:
        return None
    return C.c_void_p(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))


LBM_NN_CONV_MMA_SYNC = 0
LBM_NN_CONV_TCGEN05 = 1
LBM_NN_CONV_AUTO = 2


def lbm_nn_set_conv_impl(impl: int) -> None:
    _check(load().lbm_nn_set_conv_impl(int(impl)))


def lbm_nn_get_conv_impl() -> int:
    return int(load().lbm_nn_get_conv_impl())


def lbm_nn_sync_status(stream=None) -> None:
    _check(load().lbm_nn_sync_status(stream))


def lbm_nn_conv_fwd(x, n, h, w, cin, wts, bias, taps, cout, relu, out, out_f32=None, stream=None):
    _check(load().lbm_nn_conv_fwd(_dp(x), n, h, w, cin, _dp(wts), _dp(bias), taps, cout, int(relu),
                                  _dp(out), _dp(out_f32), stream))


def lbm_nn_conv_bwd_data(gout, n, h, w, cout, wts, taps, cin, wflip, gin, stream=None):
    _check(load().lbm_nn_conv_bwd_data(_dp(gout), n, h, w, cout, _dp(wts), taps, cin, _dp(wflip), _dp(gin),
                                       stream))


def lbm_nn_conv_bwd_weight(x, gout, n, h, w, cin, cout, taps, dw, db, accumulate, scratch, scratch_floats,
                           stream=None):
    _check(load().lbm_nn_conv_bwd_weight(_dp(x), _dp(gout), n, h, w, cin, cout, taps, _dp(dw), _dp(db),
                                         int(accumulate), _dp(scratch), int(scratch_floats), stream))


def lbm_nn_relu_bwd(y, gy, gx, count, stream=None):
    _check(load().lbm_nn_relu_bwd(_dp(y), _dp(gy), _dp(gx), int(count), stream))


def lbm_nn_pool2_fwd(x, n, h, w, c, out, stream=None):
    _check(load().lbm_nn_pool2_fwd(_dp(x), n, h, w, c, _dp(out), stream))


def lbm_nn_pool2_bwd(gout, n, h, w, c, gin, stream=None):
    _check(load().lbm_nn_pool2_bwd(_dp(gout), n, h, w, c, _dp(gin), stream))


def lbm_nn_up2_fwd(x, n, h, w, c, out, stream=None):
    _check(load().lbm_nn_up2_fwd(_dp(x), n, h, w, c, _dp(out), stream))


def lbm_nn_up2_bwd(gout, n, h, w, c, gin, stream=None):
    _check(load().lbm_nn_up2_bwd(_dp(gout), n, h, w, c, _dp(gin), stream))


def lbm_nn_copy_channels(src, sld, sc0, dst, dld, dc0, nc, npix, stream=None):
    _check(load().lbm_nn_copy_channels(_dp(src), sld, sc0, _dp(dst), dld, dc0, nc, int(npix), stream))


def lbm_nn_mse(pred, ld, target, solid, npix, nout, inv_count, grad, scratch256, loss, stream=None,
               weights=None):
    wts = None if weights is None else (C.c_float * nout)(*[float(v) for v in weights])
    _check(load().lbm_nn_mse(_dp(pred), ld, _dp(target), _dp(solid), int(npix), nout, wts, float(inv_count),
                             _dp(grad), _dp(scratch256), _dp(loss), stream))


def lbm_nn_adamw(p, g, m, v, n, lr, b1, b2, eps, wd, step, p_bf16=None, stream=None):
    _check(load().lbm_nn_adamw(_dp(p), _dp(g), _dp(m), _dp(v), int(n), lr, b1, b2, eps, wd, int(step),
                               _dp(p_bf16), stream))


def lbm_nn_add(a, b, out, n, stream=None):
    _check(load().lbm_nn_add(_dp(a), _dp(b), _dp(out), int(n), stream))


def lbm_nn_f32_to_bf16(a, b, n, stream=None):
    _check(load().lbm_nn_f32_to_bf16(_dp(a), _dp(b), int(n), stream))


def lbm_nn_make_input(solid, h, w, tau_feat, out, stream=None):
    _check(load().lbm_nn_make_input(_dp(solid), h, w, float(tau_feat), _dp(out), stream))


def lbm_nn_targets(s: Solver, d: int, out) -> None:
    _check(load().lbm_nn_targets(s.handle, d, _dp(out)), s.handle)


def lbm_warm_start(s: Solver, d: int, pred, ld: int) -> None:
    _check(load().lbm_warm_start(s.handle, d, _dp(pred), ld), s.handle)


def lbm_get_step(s: Solver) -> int:
    v = C.c_int64()
    _check(load().lbm_get_step(s.handle, C.byref(v)), s.handle)
    return v.value


def lbm_save(s: Solver, path: str) -> None:
    _check(load().lbm_save(s.handle, path.encode()), s.handle)


def lbm_load(path: str, masks=None, options: Optional[lbm_options] = None) -> Solver:
    o = options or make_options()
    h = C.c_void_p()
    _check(load().lbm_load(path.encode(), C.byref(o), C.byref(h)))
    return Solver(h, masks if masks is not None else [], [], [], o)
