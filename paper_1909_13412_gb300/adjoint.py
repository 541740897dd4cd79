"""Differentiable coupled runs: a ``torch.autograd.Function`` over liblbp's adjoint.

``trajectory(...)`` runs the coupled LBM + Stokeslet-fit Langevin method for a
number of steps on the GPU and returns the particle velocity and position
trajectories (V^{n+1}, r^{n+1} after every step n) as CUDA tensors.  Any
PyTorch loss written on them -- a relaxation curve, a VACF -- back-propagates
through the run by the library's hand-written adjoint (``lbp_adjoint_record``
/ ``lbp_adjoint_backward``): gradients reach the relaxation time tau (and so
the viscosity nu = (tau - 1/2)/3 of Eq. 16), each particle's friction
coefficient gamma, radius R and mass M, the temperature kT, the initial
velocities and positions and the initial populations.  The forward run keeps
a checkpoint every ``checkpoint_every`` steps; the backward pass re-runs one
segment at a time from its checkpoint.

``batch_trajectory(...)`` does the same for an ensemble of independent boxes
of different sizes, each with its own relaxation time, held in one batched
handle (the realisations whose VACFs Section 3 averages): one lattice launch
and one particle launch per step and per adjoint step, a tau gradient per box.

The glue here only moves tensors and calls the C ABI; all arithmetic of the
forward and adjoint steps runs in the library's CUDA kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import lbp


@dataclass(frozen=True)
class RunSpec:
    """Everything of a run that is not differentiated."""
    nx: int
    ny: int
    nz: int
    steps: int
    checkpoint_every: int = 100
    kT_seed: int = 0
    mode: int = lbp.LBP_STOKESLET
    exclude_inside: int = 0
    precision: int = lbp.LBP_F32


@dataclass(frozen=True)
class BatchSpec:
    """The non-differentiated part of a batched run: the boxes (nx, ny, nz),
    how many particles each holds (the particle tensors list box 0's first,
    then box 1's, ...), and the run settings of RunSpec."""
    boxes: tuple
    counts: tuple
    steps: int
    checkpoint_every: int = 100
    kT_seed: int = 0
    mode: int = lbp.LBP_STOKESLET
    exclude_inside: int = 0
    precision: int = lbp.LBP_F32

    @property
    def nodes(self):
        return sum(nx * ny * nz for nx, ny, nz in self.boxes)


def _dev(x):
    return x.detach().to(device="cuda", dtype=torch.float64).contiguous()


class Run(torch.autograd.Function):
    """(tau, kT, gamma, radius, mass, v0, r0, f0) -> (V trajectory, r trajectory);
    spec is a RunSpec (one box, scalar tau) or a BatchSpec (an ensemble of
    boxes in one handle, tau one per box)."""

    @staticmethod
    def forward(ctx, tau, kT, gamma, radius, mass, v0, r0, f0, f_ext, pinned, spec: RunSpec):
        n = r0.shape[0]
        batched = isinstance(spec, BatchSpec)
        if batched:
            taus = tau.detach().reshape(-1).tolist()
            if len(taus) != len(spec.boxes) or len(spec.counts) != len(spec.boxes) or sum(spec.counts) != n:
                raise ValueError("tau needs one entry per box and counts must add up to the particles")
            h = lbp.lbp_create_batch([(nx, ny, nz, t) for (nx, ny, nz), t in zip(spec.boxes, taus)],
                                     precision=spec.precision)
        else:
            h = lbp.lbp_create(spec.nx, spec.ny, spec.nz, float(tau), precision=spec.precision)
        try:
            if f0 is not None:
                lbp.lbp_set_populations(h, _dev(f0).reshape(-1))
            if n:
                r, v, m, g, R = _dev(r0), _dev(v0), _dev(mass), _dev(gamma), _dev(radius)
                if batched:
                    p0 = 0
                    for b, nb in enumerate(spec.counts):
                        if nb:
                            sl = slice(p0, p0 + nb)
                            lbp.lbp_particles_add_to(h, b, r[sl], v[sl], m[sl], g[sl], R[sl])
                        p0 += nb
                else:
                    lbp.lbp_particles_add(h, r, v, m, g, R)
                lbp.lbp_particles_set_params(h, kT=float(kT), seed=spec.kT_seed, mode=spec.mode,
                                             fit_exclude_inside=spec.exclude_inside)
                if f_ext is not None or pinned is not None:
                    lbp.lbp_particles_set_external_force(
                        h, None if f_ext is None else _dev(f_ext),
                        None if pinned is None else pinned.detach().to(device="cuda", dtype=torch.uint8).contiguous())
            vt = torch.empty((spec.steps, n, 3), dtype=torch.float64, device="cuda")
            rt = torch.empty((spec.steps, n, 3), dtype=torch.float64, device="cuda")
            lbp.lbp_adjoint_record(h, spec.steps, spec.checkpoint_every, vt, rt)
        except Exception:
            lbp.lbp_destroy(h)
            raise
        ctx.h = h
        ctx.spec = spec
        ctx.n = n
        ctx.inputs = [(x.device, x.dtype, x.shape) if isinstance(x, torch.Tensor) else None
                      for x in (tau, kT, gamma, radius, mass, v0, r0, f0)]
        return vt, rt

    @staticmethod
    def backward(ctx, g_v, g_r):
        h, spec, n = ctx.h, ctx.spec, ctx.n
        names = ("tau", "kT", "gamma", "radius", "mass", "v0", "r0", "f0")
        ntau = len(spec.boxes) if isinstance(spec, BatchSpec) else 1
        shapes = {"tau": (ntau,), "kT": (1,), "gamma": (n,), "radius": (n,), "mass": (n,),
                  "v0": (n, 3), "r0": (n, 3), "f0": (15, h.N)}
        out = {}
        for i, name in enumerate(names):
            if ctx.needs_input_grad[i] and ctx.inputs[i] is not None:
                out[name] = torch.empty(shapes[name], dtype=torch.float64, device="cuda")
        gv = None if g_v is None else g_v.to(device="cuda", dtype=torch.float64).contiguous()
        gr = None if g_r is None else g_r.to(device="cuda", dtype=torch.float64).contiguous()
        try:
            if out:
                lbp.lbp_adjoint_backward(h, spec.steps, gv, gr, out)
        finally:
            lbp.lbp_destroy(h)
            ctx.h = None
        grads = []
        for i, name in enumerate(names):
            if name in out:
                dev, dt, shape = ctx.inputs[i]
                grads.append(out[name].reshape(shape).to(device=dev, dtype=dt))
            else:
                grads.append(None)
        return (*grads, None, None, None)


def trajectory(tau, gamma, radius, mass, v0, r0, spec: RunSpec, kT=0.0, f0=None, f_ext=None,
               pinned=None):
    """V and r trajectories ([steps, n, 3] CUDA FP64) of a run, differentiable
    with respect to every tensor argument (tau, kT scalars; gamma, radius, mass
    [n]; v0, r0 [n, 3]; f0 [15, nz, ny, nx] post-collision populations, rest
    state if None).  f_ext ([n, 3] external forces) and pinned ([n] flags) are
    held fixed."""
    if not isinstance(kT, torch.Tensor):
        kT = torch.tensor(float(kT), dtype=torch.float64)
    if not isinstance(tau, torch.Tensor):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    return Run.apply(tau, kT, gamma, radius, mass, v0, r0, f0, f_ext, pinned, spec)


def batch_trajectory(tau, gamma, radius, mass, v0, r0, spec: BatchSpec, kT=0.0, f0=None, f_ext=None,
                     pinned=None):
    """V and r trajectories ([steps, n, 3] CUDA FP64, particles in box order) of
    a batched run, differentiable with respect to tau ([number of boxes], one
    relaxation time per box), kT, the per-particle gamma, radius, mass [n],
    v0, r0 [n, 3] and f0 ([15, total nodes], the boxes' nodes one after another,
    each box in z, y, x order; rest state if None).  A random force, if kT > 0,
    is keyed by the particle's index in the whole batch."""
    if not isinstance(kT, torch.Tensor):
        kT = torch.tensor(float(kT), dtype=torch.float64)
    if not isinstance(tau, torch.Tensor):
        tau = torch.tensor([float(t) for t in tau], dtype=torch.float64)
    return Run.apply(tau, kT, gamma, radius, mass, v0, r0, f0, f_ext, pinned, spec)


def stokes_radius(gamma, tau, rho0=1.0):
    """R with gamma = 6 pi rho0 nu R, nu = (tau - 1/2)/3 (Stokes' law, Eq. 16);
    differentiable, so a run whose R follows Stokes' law gets the chain rule."""
    return gamma / (6.0 * math.pi * rho0 * (tau - 0.5) / 3.0)


def relaxation_loss(v_traj, v0, t_relax):
    """Mean squared deviation of the velocity relaxation V_i(t) from the target
    exponential V_i(0) exp(-t / t_relax), t = 1..steps."""
    steps = v_traj.shape[0]
    t = torch.arange(1, steps + 1, dtype=v_traj.dtype, device=v_traj.device)
    target = v0.to(v_traj)[None] * torch.exp(-t / t_relax)[:, None, None]
    return ((v_traj - target) ** 2).mean()


def vacf(v_traj, max_lag):
    """C(k) = mean over particles and origins of V(t0).V(t0 + k), k = 0..max_lag
    (the estimator of Section 3; differentiable).

    All lags at once through the correlation theorem: the summed
    autocorrelation of every particle component is the inverse real FFT of
    the summed power spectra of the trajectory zero-padded to a length
    >= T + max_lag (no wrap-around), divided by the number of (origin,
    particle) pairs at each lag.  In FP64 its rounding error is ~1e-16 of C(0)."""
    T, n = v_traj.shape[0], v_traj.shape[1]
    K = int(max_lag)
    if K < 0 or K >= T:
        raise ValueError("max_lag must lie in [0, number of samples)")
    nfft = 1 << (T + K - 1).bit_length()
    X = torch.fft.rfft(v_traj.reshape(T, -1), n=nfft, dim=0)
    power = (X.real ** 2 + X.imag ** 2).sum(1)
    corr = torch.fft.irfft(power, n=nfft)[:K + 1]
    pairs = (T - torch.arange(K + 1, dtype=v_traj.dtype, device=v_traj.device)) * n
    return corr / pairs
