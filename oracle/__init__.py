"""FP64 CPU oracle of the LBM + Stokeslet-fit Langevin step (arXiv:1909.13412).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA library.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
and ``--impl reference`` legs) may import it.  It shares no code with the CUDA
path: the arithmetic lives in ``lbp_oracle.c``, written from Section 2 of the
paper, and this module only marshals numpy arrays through ctypes.

Every function cites the passage it follows; the C file states the step order
and every reading of the paper it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbp_oracle.c")
_LIB = os.path.join(_HERE, "liblbp_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 15
STOKESLET, POINTWISE, BROWNIAN = 0, 1, 2

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``lbp_oracle.c`` with gcc (FP64, FMA contraction off, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                   "-fopenmp", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """ctypes handle of a compiled oracle library at `path`, with every signature set."""
    L = C.CDLL(path)
    vp = C.c_void_p
    L.or_d3q15.argtypes = [_i32p, _dp]
    L.or_stream.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int]
    L.or_moments.argtypes = [_dp, _dp, _dp, C.c_int64]
    L.or_feq.argtypes = [C.c_double, _dp, _dp]
    L.or_collide.argtypes = [_dp, _dp, _dp, vp, C.c_double, C.c_int64, _dp]
    L.or_collide_dev.argtypes = [_dp, _dp, _dp, vp, C.c_double, C.c_int64, _dp]
    L.or_set_deviation.argtypes = [vp, C.c_int]
    L.or_set_body_force.argtypes = [vp, _dp]
    L.or_corners.argtypes = [_dp, _i32p, _dp, _dp]
    L.or_stokeslet_fit.argtypes = [_dp, _dp, _dp, C.c_double, C.c_int, _dp]
    L.or_stokeslet_fit.restype = C.c_double
    L.or_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
    L.or_noise_xi.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, _dp]
    L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double]
    L.or_create.restype = vp
    L.or_destroy.argtypes = [vp]
    L.or_set_fhat.argtypes = [vp, _dp]
    L.or_get_fhat.argtypes = [vp, _dp]
    L.or_set_step.argtypes = [vp, C.c_int64]
    L.or_get_step.argtypes = [vp]
    L.or_get_step.restype = C.c_int64
    L.or_get_fields.argtypes = [vp, _dp, _dp, vp]
    L.or_add_particles.argtypes = [vp, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.or_set_params.argtypes = [vp, C.c_double, C.c_uint64, C.c_int, C.c_int]
    L.or_set_external.argtypes = [vp, vp, vp]
    L.or_set_particles.argtypes = [vp, vp, vp]
    L.or_get_particles.argtypes = [vp, vp, vp, vp, vp]
    L.or_step.argtypes = [vp, C.c_int64]
    L.or_spread_only.argtypes = [vp, _dp]
    L.or_vacf.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, C.c_int, _dp, _i64p]
    L.or_msd.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, _dp, _i64p]
    L.or_num_threads.restype = C.c_int
    L.or_set_num_threads.argtypes = [C.c_int]
    L.or_set_num_threads.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = bind(_LIB)
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- tables
def d3q15():
    """D3Q15 velocity set e [15,3] and weights w [15] (Section 2.2)."""
    e = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    lib().or_d3q15(e.reshape(-1), w)
    return e, w


# ---------------------------------------------------------------- lattice pieces
def stream(fhat):
    """Eq. 20 in pull form on a periodic box; fhat is [15, nz, ny, nx]."""
    fhat = _c(fhat)
    _, nz, ny, nx = fhat.shape
    f = np.empty_like(fhat)
    lib().or_stream(fhat.reshape(-1), f.reshape(-1), nx, ny, nz)
    return f


def moments(f):
    """Eqs. 12-13: rho~ [N...] and u [3, N...] of f [15, ...]."""
    f = _c(f)
    shp = f.shape[1:]
    N = int(np.prod(shp))
    rho = np.empty(N)
    u = np.empty(3 * N)
    lib().or_moments(f.reshape(-1), rho, u, N)
    return rho.reshape(shp), u.reshape((3,) + shp)


def feq(rho, u):
    """Eq. 17 at one node."""
    out = np.empty(Q)
    lib().or_feq(float(rho), _c(u), out)
    return out


def collide(f, rho, u, tau, F=None):
    """Eqs. 14-15, 18-19: post-collision fhat from f, its moments and force F."""
    f = _c(f)
    shp = f.shape[1:]
    N = int(np.prod(shp))
    out = np.empty_like(f)
    Fc = None if F is None else _c(F)
    lib().or_collide(f.reshape(-1), _c(rho).reshape(-1), _c(u).reshape(-1), _ptr(Fc),
                     float(tau), N, out.reshape(-1))
    return out


def corners(r):
    """Cell base, corner offsets d_p = x_p - r [8,3] and trilinear weights W_p [8]."""
    base = np.zeros(3, np.int32)
    d = np.zeros(24)
    Wp = np.zeros(8)
    lib().or_corners(_c(r), base, d, Wp)
    return base, d.reshape(8, 3), Wp


def stokeslet_fit(d, uN, V, R, exclude_inside=False):
    """Eq. 8 least-squares fit: returns (U_inf, e^N)."""
    eN = np.zeros(3)
    U = lib().or_stokeslet_fit(_c(d).reshape(-1), _c(uN).reshape(-1), _c(V), float(R),
                               int(exclude_inside), eN)
    return U, eN


def philox4x64_10(ctr, key):
    """Philox-4x64-10 block function (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64_10(_c(ctr, np.uint64), _c(key, np.uint64), out)
    return out


def noise_xi(seed, step, pid):
    """Unit-variance uniform random-force numbers of (step, particle)."""
    xi = np.zeros(3)
    lib().or_noise_xi(int(seed), int(step), int(pid), xi)
    return xi


def vacf(Vtraj, K, stride=1):
    """VACF sums C(k) = sum_{i,t0} V_i(t0).V_i(t0+k) and pair counts."""
    V = _c(Vtraj)
    T, npart, _ = V.shape
    cs = np.zeros(K + 1)
    cnt = np.zeros(K + 1, np.int64)
    lib().or_vacf(V.reshape(-1), T, npart, K, stride, cs, cnt)
    return cs, cnt


def msd(Xtraj, K):
    """Mean squared displacement sums M(k) = sum_{i,t0} |X_i(t0+k) - X_i(t0)|^2
    of unwrapped positions X [T, n, 3], and pair counts."""
    X = _c(Xtraj)
    T, npart, _ = X.shape
    ms = np.zeros(K + 1)
    cnt = np.zeros(K + 1, np.int64)
    lib().or_msd(X.reshape(-1), T, npart, K, ms, cnt)
    return ms, cnt


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    """OpenMP threads of the oracle's loops over z-planes (timing only)."""
    lib().or_set_num_threads(int(n))


# ---------------------------------------------------------------- whole system
class Sim:
    """Periodic LBM box with Langevin particles; one ``step`` = one time step."""

    def __init__(self, nx, ny, nz, tau, library=None, deviation=False):
        """``library``: another compiled copy of the oracle (``bind``), used by the
        tests that check that a pin fails when a mistake is planted in a copy.
        ``deviation``: keep and step the state as g = fhat - w_a (the same
        method, a self-check of the deviation algebra); fhat in and out stays
        the full population."""
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.tau = tau
        self.np = 0
        self._L = library if library is not None else lib()
        self._h = self._L.or_create(nx, ny, nz, float(tau))
        self._L.or_set_deviation(self._h, int(bool(deviation)))

    def close(self):
        if self._h:
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fhat(self, fhat):
        self._L.or_set_fhat(self._h, _c(fhat).reshape(-1))

    def fhat(self):
        out = np.empty((Q,) + self.shape)
        self._L.or_get_fhat(self._h, out.reshape(-1))
        return out

    def set_step(self, n):
        self._L.or_set_step(self._h, int(n))

    @property
    def step_index(self):
        return self._L.or_get_step(self._h)

    def fields(self):
        rho = np.empty(self.N)
        u = np.empty(3 * self.N)
        p = np.empty(self.N)
        self._L.or_get_fields(self._h, rho, u, _ptr(p))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape), p.reshape(self.shape)

    def add_particles(self, r, V, M, gamma, R):
        r, V = _c(r).reshape(-1, 3), _c(V).reshape(-1, 3)
        n = r.shape[0]
        M, gamma, R = (_c(np.broadcast_to(x, (n,))) for x in (M, gamma, R))
        self._L.or_add_particles(self._h, n, r.reshape(-1), V.reshape(-1), M, gamma, R)
        self.np += n

    def set_params(self, kT=0.0, seed=0, mode=STOKESLET, exclude_inside=False):
        self._L.or_set_params(self._h, float(kT), int(seed), int(mode), int(exclude_inside))

    def set_external(self, Fext=None, pinned=None):
        F = None if Fext is None else _c(Fext).reshape(-1)
        P = None if pinned is None else _c(pinned, np.uint8)
        self._L.or_set_external(self._h, _ptr(F), _ptr(P))

    def set_body_force(self, G):
        """Uniform external force density on every node (the F of Eq. 18)."""
        self._L.or_set_body_force(self._h, _c(G).reshape(3))

    def set_particles(self, r=None, V=None):
        rr = None if r is None else _c(r).reshape(-1)
        vv = None if V is None else _c(V).reshape(-1)
        self._L.or_set_particles(self._h, _ptr(rr), _ptr(vv))

    def particles(self):
        r = np.empty((self.np, 3))
        V = np.empty((self.np, 3))
        FH = np.empty((self.np, 3))
        FR = np.empty((self.np, 3))
        self._L.or_get_particles(self._h, _ptr(r), _ptr(V), _ptr(FH), _ptr(FR))
        return r, V, FH, FR

    def step(self, n=1):
        self._L.or_step(self._h, int(n))

    def spread_only(self):
        F = np.empty(3 * self.N)
        self._L.or_spread_only(self._h, F)
        return F.reshape((3,) + self.shape)
