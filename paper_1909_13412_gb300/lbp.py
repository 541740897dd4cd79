"""Thin ctypes binding of liblbp (include/lbp.h), with the C function names.

Argument marshalling only: every step of the method runs in the CUDA kernels
of liblbp.so.  Arrays may be numpy arrays (host memory, ``on_device=0``) or
CUDA torch tensors (device memory, ``on_device=1``); the binding checks dtype,
size and contiguity, passes the raw pointer and raises ``LbpError`` on any
non-zero status.  If liblbp.so has not been built the import of a function
raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbp.so")

LBP_OK, LBP_EINVAL, LBP_ENOMEM, LBP_ECUDA, LBP_ETIMEOUT, LBP_ENAN, LBP_ESTATE, LBP_ERANGE = range(8)
LBP_F32, LBP_BF16, LBP_F16 = 0, 1, 2
LBP_STOKESLET, LBP_POINTWISE, LBP_BROWNIAN = 0, 1, 2
Q = 15

_STATUS_NAMES = {0: "LBP_OK", 1: "LBP_EINVAL", 2: "LBP_ENOMEM", 3: "LBP_ECUDA", 4: "LBP_ETIMEOUT",
                 5: "LBP_ENAN", 6: "LBP_ESTATE", 7: "LBP_ERANGE"}


class LbpError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lbp_lattice_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("tau", C.c_double),
                ("precision", C.c_int)]


class lbp_particle_params(C.Structure):
    _fields_ = [("kT", C.c_double), ("seed", C.c_uint64), ("mode", C.c_int),
                ("fit_exclude_inside", C.c_int)]


_vp = C.c_void_p
_SIGS = {
    "lbp_create": [C.POINTER(lbp_lattice_desc), _vp, C.POINTER(_vp)],
    "lbp_destroy": [_vp],
    "lbp_create_batch": [_vp, C.c_int, _vp, C.POINTER(_vp)],
    "lbp_replica_info": [_vp, C.c_int, _vp, _vp, _vp],
    "lbp_replica_count": [_vp, C.POINTER(C.c_int)],
    "lbp_particles_add_to": [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int],
    "lbp_set_populations": [_vp, _vp, C.c_int],
    "lbp_read_populations": [_vp, _vp, C.c_int],
    "lbp_read_fields": [_vp, _vp, _vp, _vp, C.c_int],
    "lbp_particles_add": [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int],
    "lbp_particles_set_params": [_vp, C.POINTER(lbp_particle_params)],
    "lbp_particles_set_external_force": [_vp, _vp, _vp, C.c_int],
    "lbp_particles_set_state": [_vp, _vp, _vp, C.c_int],
    "lbp_particles_read": [_vp, _vp, _vp, _vp, _vp, C.c_int],
    "lbp_particles_read_cells": [_vp, _vp, _vp, C.c_int],
    "lbp_particles_count": [_vp, C.POINTER(C.c_int)],
    "lbp_volume_fraction": [_vp, C.c_int, C.POINTER(C.c_double)],
    "lbp_step": [_vp, C.c_int64],
    "lbp_set_step_index": [_vp, C.c_int64],
    "lbp_get_step_index": [_vp, C.POINTER(C.c_int64)],
    "lbp_vacf_configure": [_vp, C.c_int],
    "lbp_vacf_read": [_vp, _vp, _vp, C.c_int],
    "lbp_msd_read": [_vp, _vp, _vp, C.c_int],
    "lbp_vacf_configure_ex": [_vp, C.c_int, C.c_int],
    "lbp_autotune": [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "lbp_set_block_shape": [_vp, C.c_int, C.c_int],
    "lbp_step_exchange": [_vp, _vp, _vp, _vp, C.c_int],
    "lbp_adjoint_record": [_vp, C.c_int64, C.c_int, _vp, _vp, C.c_int],
    "lbp_adjoint_backward": [_vp, _vp, _vp, C.c_int, _vp],
    "lbp_set_block_rows": [_vp, C.c_int],
    "lbp_set_body_force": [_vp, C.c_int, _vp],
    "lbp_set_fluid": [_vp, _vp, _vp, C.c_int],
    "lbp_vacf_read_per_particle": [_vp, _vp, _vp, C.c_int],
    "lbp_check": [_vp],
    "lbp_budget_track": [_vp, C.c_int],
    "lbp_budget": [_vp, _vp],
    "lbp_set_wait_bound": [_vp, C.c_int64],
    "lbp_set_wait_probe": [_vp, C.c_int],
    "lbp_checkpoint_size": [_vp, C.POINTER(C.c_size_t)],
    "lbp_checkpoint_save": [_vp, _vp, C.c_int],
    "lbp_checkpoint_load": [_vp, _vp, C.c_int],
    "lbp_set_use_graphs": [_vp, C.c_int],
    "lbp_diagnostics": [_vp, _vp, C.c_int],
    "lbp_timing_enable": [_vp, C.c_int],
    "lbp_timing_read": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)],
    "lbp_philox4x64_10": [_vp, _vp, _vp, C.c_int64, _vp],
    "lbp_vacf_correlate_noalloc": [_vp, C.c_int64, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp],
}

_lib = None


def load():
    """Load liblbp.so; raise if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        for name, argtypes in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = argtypes
            fn.restype = C.c_int
        lib.lbp_last_error.argtypes = []
        lib.lbp_last_error.restype = C.c_char_p
        lib.lbp_version.argtypes = []
        lib.lbp_version.restype = C.c_int
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS) + ["lbp_last_error", "lbp_version"]


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != LBP_OK:
        raise LbpError(st, name, lib.lbp_last_error().decode())
    return st


# ------------------------------------------------------------------ marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype, count, name, writable=False):
    """(pointer, on_device) of a numpy array or torch tensor of `count` elements."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tmap = {np.float64: (torch.float64,), np.int64: (torch.int64,), np.float32: (torch.float32,),
                np.uint64: (torch.int64, getattr(torch, "uint64", torch.int64)),
                np.uint8: (torch.uint8,), np.int32: (torch.int32,)}
        if x.dtype not in tmap[dtype]:
            raise TypeError(f"{name}: expected {tmap[dtype][0]}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if count is not None and x.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {x.numel()}")
        return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name}: expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if writable and not a.flags.writeable:
        raise ValueError(f"{name}: array is read-only")
    if count is not None and a.size != count:
        raise ValueError(f"{name}: expected {count} elements, got {a.size}")
    return C.c_void_p(a.ctypes.data), 0


def _same_side(*pairs):
    sides = {d for _, d in pairs if d is not None}
    if len(sides) > 1:
        raise ValueError("all arrays of one call must be on the same side (host or device)")
    return sides.pop() if sides else 0


class Handle:
    """Owning wrapper of an lbp_sim* with its sizes (the C calls stay the API)."""

    def __init__(self, ptr, nx, ny, nz):
        self.ptr = ptr
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz

    @property
    def np(self):
        n = C.c_int()
        _call("lbp_particles_count", self.ptr, C.byref(n))
        return n.value

    def close(self):
        if self.ptr:
            lbp_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ the C calls
def lbp_version() -> int:
    return load().lbp_version()


def lbp_last_error() -> str:
    return load().lbp_last_error().decode()


def lbp_create(nx, ny, nz, tau, precision=LBP_F32, stream=None) -> Handle:
    desc = lbp_lattice_desc(int(nx), int(ny), int(nz), float(tau), int(precision))
    out = C.c_void_p()
    s = C.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0))
    _call("lbp_create", C.byref(desc), s, C.byref(out))
    return Handle(out, int(nx), int(ny), int(nz))


def lbp_create_batch(boxes, precision=LBP_F32, stream=None) -> Handle:
    """boxes: sequence of (nx, ny, nz, tau).  The handle's N is the total node count."""
    arr = (lbp_lattice_desc * len(boxes))(*[lbp_lattice_desc(int(a), int(b), int(c), float(t),
                                                             int(precision)) for a, b, c, t in boxes])
    out = C.c_void_p()
    s = C.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0))
    _call("lbp_create_batch", C.cast(arr, C.c_void_p), len(boxes), s, C.byref(out))
    h = Handle(out, 0, 0, 0)
    h.N = sum(int(a) * int(b) * int(c) for a, b, c, _ in boxes)
    h.boxes = [tuple(bx) for bx in boxes]
    return h


def lbp_replica_info(h: Handle, replica):
    dims = (C.c_int * 3)()
    tau = C.c_double()
    off = C.c_int64()
    _call("lbp_replica_info", h.ptr, int(replica), C.cast(dims, C.c_void_p), C.byref(tau), C.byref(off))
    return (dims[0], dims[1], dims[2]), tau.value, off.value


def lbp_replica_count(h: Handle) -> int:
    n = C.c_int()
    _call("lbp_replica_count", h.ptr, C.byref(n))
    return n.value


def lbp_particles_add_to(h: Handle, replica, r, v, mass, gamma, radius=None):
    n = (r.numel() if _is_torch(r) else r.size) // 3
    args = [_ptr(r, np.float64, 3 * n, "r"), _ptr(v, np.float64, 3 * n, "v"),
            _ptr(mass, np.float64, n, "mass"), _ptr(gamma, np.float64, n, "gamma"),
            _ptr(radius, np.float64, n, "radius")]
    d = _same_side(*args)
    _call("lbp_particles_add_to", h.ptr, int(replica), n, *[a[0] for a in args], d)
    _warn_if_dense(h)


def lbp_destroy(h: Handle):
    if h.ptr:
        _call("lbp_destroy", h.ptr)
        h.ptr = None


def lbp_set_populations(h: Handle, f):
    p, d = _ptr(f, np.float64, Q * h.N, "f")
    _call("lbp_set_populations", h.ptr, p, d)


def lbp_set_fluid(h: Handle, rho=None, u=None):
    """Set every node to f^eq(rho~, u) (Eq. 17); rho [N], u [3, N] FP64 or None."""
    a = _ptr(rho, np.float64, h.N, "rho")
    b = _ptr(u, np.float64, 3 * h.N, "u")
    d = _same_side(a, b)
    _call("lbp_set_fluid", h.ptr, a[0], b[0], d)


def lbp_read_populations(h: Handle, f):
    p, d = _ptr(f, np.float64, Q * h.N, "f", writable=True)
    _call("lbp_read_populations", h.ptr, p, d)
    return f


def lbp_read_fields(h: Handle, rho=None, u=None, p=None):
    a = _ptr(rho, np.float64, h.N, "rho", True)
    b = _ptr(u, np.float64, 3 * h.N, "u", True)
    c = _ptr(p, np.float64, h.N, "p", True)
    d = _same_side(a, b, c)
    _call("lbp_read_fields", h.ptr, a[0], b[0], c[0], d)


def lbp_particles_add(h: Handle, r, v, mass, gamma, radius=None):
    n = (r.numel() if _is_torch(r) else r.size) // 3
    args = [_ptr(r, np.float64, 3 * n, "r"), _ptr(v, np.float64, 3 * n, "v"),
            _ptr(mass, np.float64, n, "mass"), _ptr(gamma, np.float64, n, "gamma"),
            _ptr(radius, np.float64, n, "radius")]
    d = _same_side(*args)
    _call("lbp_particles_add", h.ptr, n, *[a[0] for a in args], d)
    _warn_if_dense(h)


# the volume fraction below which the method was checked (Section 2.2)
PHI_CHECKED = 0.1


def lbp_volume_fraction(h: Handle, replica=-1) -> float:
    phi = C.c_double()
    _call("lbp_volume_fraction", h.ptr, int(replica), C.byref(phi))
    return phi.value


def _warn_if_dense(h: Handle):
    phi = lbp_volume_fraction(h)
    if phi > PHI_CHECKED:
        warnings.warn(f"particle volume fraction {phi:.3f} exceeds {PHI_CHECKED}, the range the "
                      "method was checked for (Section 2.2)", RuntimeWarning, stacklevel=3)


def lbp_particles_set_params(h: Handle, kT=0.0, seed=0, mode=LBP_STOKESLET, fit_exclude_inside=0):
    prm = lbp_particle_params(float(kT), int(seed), int(mode), int(fit_exclude_inside))
    _call("lbp_particles_set_params", h.ptr, C.byref(prm))


def lbp_particles_set_external_force(h: Handle, f_ext=None, pinned=None):
    n = h.np
    a = _ptr(f_ext, np.float64, 3 * n, "f_ext")
    b = _ptr(pinned, np.uint8, n, "pinned")
    d = _same_side(a, b)
    _call("lbp_particles_set_external_force", h.ptr, a[0], b[0], d)


def lbp_particles_set_state(h: Handle, r=None, v=None):
    n = h.np
    a = _ptr(r, np.float64, 3 * n, "r")
    b = _ptr(v, np.float64, 3 * n, "v")
    d = _same_side(a, b)
    _call("lbp_particles_set_state", h.ptr, a[0], b[0], d)


def lbp_particles_read(h: Handle, r=None, v=None, f_h=None, f_r=None):
    n = h.np
    args = [_ptr(x, np.float64, 3 * n, nm, True) for x, nm in ((r, "r"), (v, "v"), (f_h, "f_h"), (f_r, "f_r"))]
    d = _same_side(*args)
    _call("lbp_particles_read", h.ptr, *[a[0] for a in args], d)


def lbp_particles_read_cells(h: Handle, base, frac):
    n = h.np
    a = _ptr(base, np.int32, 3 * n, "base", True)
    b = _ptr(frac, np.float64, 3 * n, "frac", True)
    d = _same_side(a, b)
    _call("lbp_particles_read_cells", h.ptr, a[0], b[0], d)


def lbp_particles_count(h: Handle) -> int:
    return h.np


def lbp_step(h: Handle, nsteps=1):
    _call("lbp_step", h.ptr, int(nsteps))


def lbp_step_exchange(h: Handle, f_ext=None, r=None, v=None):
    """Upload external forces, advance one step, read positions and velocities
    ([n, 3] FP64 each, any may be None) -- one call, one synchronisation."""
    n = h.np
    a = _ptr(f_ext, np.float64, 3 * n, "f_ext")
    b = _ptr(r, np.float64, 3 * n, "r", True)
    c = _ptr(v, np.float64, 3 * n, "v", True)
    d = _same_side(a, b, c)
    _call("lbp_step_exchange", h.ptr, a[0], b[0], c[0], d)


def lbp_set_step_index(h: Handle, step):
    _call("lbp_set_step_index", h.ptr, int(step))


def lbp_get_step_index(h: Handle) -> int:
    v = C.c_int64()
    _call("lbp_get_step_index", h.ptr, C.byref(v))
    return v.value


def lbp_vacf_configure(h: Handle, max_lag):
    _call("lbp_vacf_configure", h.ptr, int(max_lag))


def lbp_vacf_read(h: Handle, csum, counts):
    a = _ptr(csum, np.float64, None, "csum", True)
    b = _ptr(counts, np.int64, None, "counts", True)
    d = _same_side(a, b)
    _call("lbp_vacf_read", h.ptr, a[0], b[0], d)


def lbp_msd_read(h: Handle, msum, counts):
    """Mean squared displacement sums [max_lag + 1] (FP64) and pair counts."""
    a = _ptr(msum, np.float64, None, "msum", True)
    b = _ptr(counts, np.int64, None, "counts", True)
    d = _same_side(a, b)
    _call("lbp_msd_read", h.ptr, a[0], b[0], d)


def lbp_vacf_configure_ex(h: Handle, max_lag, per_particle):
    _call("lbp_vacf_configure_ex", h.ptr, int(max_lag), int(bool(per_particle)))


def lbp_vacf_read_per_particle(h: Handle, csum, counts):
    """csum: [n_particles, max_lag + 1] FP64; counts: [max_lag + 1] int64."""
    a = _ptr(csum, np.float64, None, "csum", True)
    b = _ptr(counts, np.int64, None, "counts", True)
    d = _same_side(a, b)
    _call("lbp_vacf_read_per_particle", h.ptr, a[0], b[0], d)


class lbp_gradients(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("tau", "kT", "gamma", "radius", "mass", "v0", "r0", "f0")]


GRADIENT_NAMES = ("tau", "kT", "gamma", "radius", "mass", "v0", "r0", "f0")


def lbp_adjoint_record(h: Handle, nsteps, checkpoint_every, v_traj=None, r_traj=None):
    """Run nsteps steps, keeping checkpoints every checkpoint_every steps; v_traj,
    r_traj ([nsteps, n, 3] FP64) receive V^{n+1}, r^{n+1}."""
    cnt = int(nsteps) * h.np * 3
    a = _ptr(v_traj, np.float64, cnt, "v_traj", True)
    b = _ptr(r_traj, np.float64, cnt, "r_traj", True)
    d = _same_side(a, b)
    _call("lbp_adjoint_record", h.ptr, int(nsteps), int(checkpoint_every), a[0], b[0], d)


def lbp_adjoint_backward(h: Handle, nsteps, g_v=None, g_r=None, out=None):
    """Reverse sweep over the recording.  out: dict name -> writable array/tensor
    for any of GRADIENT_NAMES (shapes: tau [number of boxes]; kT [1]; gamma,
    radius, mass [n]; v0, r0 [n, 3]; f0 [15, N]), all on the same side as
    g_v / g_r."""
    n = h.np
    cnt = int(nsteps) * n * 3
    a = _ptr(g_v, np.float64, cnt, "g_v")
    b = _ptr(g_r, np.float64, cnt, "g_r")
    sizes = {"tau": lbp_replica_count(h), "kT": 1, "gamma": n, "radius": n, "mass": n, "v0": 3 * n,
             "r0": 3 * n, "f0": Q * h.N}
    g = lbp_gradients()
    ptrs = []
    for name, x in (out or {}).items():
        if name not in sizes:
            raise KeyError(f"unknown gradient {name!r}")
        pp = _ptr(x, np.float64, sizes[name], name, True)
        setattr(g, name, pp[0])
        ptrs.append(pp)
    d = _same_side(a, b, *ptrs)
    _call("lbp_adjoint_backward", h.ptr, a[0], b[0], d, C.byref(g))
    return out


def lbp_check(h: Handle):
    _call("lbp_check", h.ptr)


def lbp_diagnostics(h: Handle):
    out = np.zeros(6, np.int64)
    _call("lbp_diagnostics", h.ptr, C.c_void_p(out.ctypes.data), 6)
    return {"overflow_shares": int(out[0]), "record_slots": int(out[1]), "segments": int(out[2]),
            "rows_per_block": int(out[3]), "variant": int(out[4]), "fit_per_corner": bool(out[5])}


def lbp_set_body_force(h: Handle, g, replica=-1):
    arr = (C.c_double * 3)(*[float(x) for x in g])
    _call("lbp_set_body_force", h.ptr, int(replica), C.cast(arr, C.c_void_p))


def lbp_set_block_rows(h: Handle, rows):
    _call("lbp_set_block_rows", h.ptr, int(rows))


# (variant, rows) of the autotuner's candidates, in the order of its ms array
AUTOTUNE_SHAPES = ((0, 1), (0, 2), (0, 4), (1, 1), (1, 2), (1, 4), (2, 1), (3, 1), (3, 2), (3, 4))


def lbp_autotune(h: Handle, launches=20):
    """Pick the lattice kernel's shape by timing; returns (rows, variant, ms)
    with ms the mean launch times of the AUTOTUNE_SHAPES candidates, -1 where
    a candidate does not apply."""
    rows, variant = C.c_int(), C.c_int()
    ms = (C.c_double * len(AUTOTUNE_SHAPES))()
    _call("lbp_autotune", h.ptr, int(launches), C.byref(rows), C.byref(variant), ms)
    return rows.value, variant.value, list(ms)


def lbp_set_block_shape(h: Handle, rows, variant):
    _call("lbp_set_block_shape", h.ptr, int(rows), int(variant))


def lbp_set_use_graphs(h: Handle, enable):
    _call("lbp_set_use_graphs", h.ptr, int(bool(enable)))


def lbp_timing_enable(h: Handle, enable):
    _call("lbp_timing_enable", h.ptr, int(bool(enable)))


def lbp_timing_read(h: Handle):
    ms = C.c_double()
    n = C.c_int64()
    _call("lbp_timing_read", h.ptr, C.byref(ms), C.byref(n))
    return ms.value, n.value


def lbp_philox4x64_10(ctr, key, out, n, stream=None):
    """ctr [n,4], key [2], out [n,4]: 64-bit CUDA tensors (int64 holding the uint64 bits)."""
    a = _ptr(ctr, np.uint64, 4 * n, "ctr")
    b = _ptr(key, np.uint64, 2, "key")
    c = _ptr(out, np.uint64, 4 * n, "out", True)
    if {a[1], b[1], c[1]} != {1}:
        raise ValueError("lbp_philox4x64_10 takes device tensors")
    s = C.c_void_p(stream.cuda_stream if stream is not None else 0)
    _call("lbp_philox4x64_10", a[0], b[0], c[0], int(n), s)


def lbp_vacf_correlate_noalloc(samples, T, ncomp, max_lag, npairs, csum, counts, stream=None):
    """VACF of a device trajectory [T][ncomp] (FP32) without device allocation."""
    a = _ptr(samples, np.float32, T * ncomp, "samples") if T > 0 else (C.c_void_p(0), 1)
    b = _ptr(csum, np.float64, max_lag + 1, "csum", True)
    c = _ptr(counts, np.int64, max_lag + 1, "counts", True)
    if {a[1], b[1], c[1]} != {1}:
        raise ValueError("lbp_vacf_correlate_noalloc takes device tensors")
    s = C.c_void_p(stream.cuda_stream if stream is not None else 0)
    _call("lbp_vacf_correlate_noalloc", a[0], int(T), int(ncomp), int(max_lag), int(npairs), b[0],
          c[0], s)


def lbp_budget_track(h: Handle, enable=True):
    _call("lbp_budget_track", h.ptr, int(bool(enable)))


def lbp_budget(h: Handle):
    """[mass, fluid momentum (3), particle momentum (3), injected momentum (3)]."""
    out = np.zeros(10)
    _call("lbp_budget", h.ptr, C.c_void_p(out.ctypes.data))
    return out


def lbp_set_wait_bound(h: Handle, cycles):
    _call("lbp_set_wait_bound", h.ptr, int(cycles))


def lbp_checkpoint_size(h: Handle) -> int:
    n = C.c_size_t()
    _call("lbp_checkpoint_size", h.ptr, C.byref(n))
    return n.value


def lbp_checkpoint_save(h: Handle, buf=None):
    """Write a checkpoint into buf (a uint8 numpy array or CUDA tensor of
    lbp_checkpoint_size bytes; None: a new numpy array) and return it."""
    if buf is None:
        buf = np.empty(lbp_checkpoint_size(h), np.uint8)
    a = _ptr(buf, np.uint8, lbp_checkpoint_size(h), "buf", True)
    _call("lbp_checkpoint_save", h.ptr, a[0], a[1])
    return buf


def lbp_checkpoint_load(h: Handle, buf):
    a = _ptr(buf, np.uint8, None, "buf")
    _call("lbp_checkpoint_load", h.ptr, a[0], a[1])


def lbp_set_wait_probe(h: Handle, enable):
    _call("lbp_set_wait_probe", h.ptr, int(bool(enable)))
