"""FP64 reference gradients of the coupled LBM + Stokeslet-fit Langevin run.

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/`` this module exists to
check the CUDA library (here: its hand-written adjoint); only ``tests/`` may
import it.  It shares nothing with the CUDA path.

The time step of Section 2 is written once more, this time with PyTorch CPU
tensor operations in FP64, so that autograd can differentiate a whole run with
respect to its inputs: the relaxation time tau (viscosity nu = (tau - 1/2)/3,
Eq. 16), each particle's friction coefficient gamma, radius R and mass M, the
initial velocities V0 and positions r0, and the initial populations.  The step
order and every reading of the paper are those of ``lbp_oracle.c``:

  1. streaming, pull form (Eq. 20): f_a(x) = fhat_a(x - e_a), periodic;
  2. moments (Eqs. 12-13): rho~ = sum_a f_a, u = sum_a e_a f_a;
  3. per particle, from u at the eight corners of the cell holding r_i: the
     Stokeslet fit of Eq. 8 (or Eq. 7 with trilinear u, or Eq. 6), F_H;
  4. random force F_R = sqrt(2 gamma kT) xi (Eqs. 4-5); xi is taken from the
     C oracle's Philox-4x64-10 stream and enters here as a constant;
  5. reaction force -F_H spread to the eight corners with trilinear weights
     of r_i^n (Eq. 9);
  6. Langevin update, dt = 1 (Eqs. 1-2): V += (F_H + F_R + F_ext)/M, r += V,
     periodic wrap;
  7. BGK collision with the body force (Eqs. 14-15, 17-19):
     fhat_a = f_a + (f^eq_a - f_a)/tau + 3 w_a F.e_a.

Where the function is not differentiable (the cell index floor(r), the
skipped corners of the fit) the derivative is that of the branch taken, as
for the CUDA adjoint.  The forward values are pinned to ``lbp_oracle.c`` and
the gradients to central finite differences of it (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import BROWNIAN, POINTWISE, STOKESLET, d3q15, noise_xi

_E_NP, _W_NP = d3q15()
E = torch.tensor(_E_NP, dtype=torch.float64)          # [15, 3]
W = torch.tensor(_W_NP, dtype=torch.float64)          # [15]
CORNERS = torch.tensor([[p & 1, (p >> 1) & 1, (p >> 2) & 1] for p in range(8)],
                       dtype=torch.float64)            # [8, 3], corner p = cx + 2 cy + 4 cz


def stream(fhat):
    """Eq. 20 (pull): f_a(x) = fhat_a(x - e_a) on the periodic [15, nz, ny, nx] grid."""
    out = []
    for a in range(15):
        ex, ey, ez = (int(v) for v in _E_NP[a])
        out.append(torch.roll(fhat[a], shifts=(ez, ey, ex), dims=(0, 1, 2)))
    return torch.stack(out)


def moments(f):
    """Eqs. 12-13: rho~ = sum_a f_a and u = sum_a e_a f_a (no 1/rho~)."""
    return f.sum(0), torch.einsum("ak,azyx->kzyx", E, f)


def feq(rho, u):
    """Eq. 17: f^eq_a = w_a [rho~ + 3 e_a.u + 9/2 (e_a.u)^2 - 3/2 u.u]."""
    eu = torch.einsum("ak,kzyx->azyx", E, u)
    uu = (u * u).sum(0)
    return W[:, None, None, None] * (rho[None] + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu[None])


def collide(f, rho, u, F, tau):
    """Eqs. 14, 15, 18, 19: fhat_a = f_a + (f^eq_a - f_a)/tau + w_a 3 F.e_a."""
    G = 3.0 * torch.einsum("ak,kzyx->azyx", E, F)
    return f + (feq(rho, u) - f) / tau + W[:, None, None, None] * G


def stokeslet_force(d, uN, V, R, gamma, exclude_inside):
    """F_H = gamma U_inf e^N from the least-squares fit of Eq. 8 (Section 2.1).

    d: [n, 8, 3] corner minus particle; uN: [n, 8, 3]; V: [n, 3]; R, gamma: [n].
    w_p = u_p - V, e^N = mean(w)/|mean(w)|, a_p = (1 - 3R/(4r)) e^N
    - 3R (e^N.d)/(4 r^3) d, U_inf = sum w.a / sum |a|^2 over the corners kept.
    """
    w = uN - V[:, None, :]
    wm = w.sum(1) / 8.0
    nw = torch.sqrt((wm * wm).sum(1))
    alive = nw.detach() > 0.0
    eN = wm / torch.where(alive, nw, torch.ones_like(nw))[:, None]
    rp = torch.sqrt((d * d).sum(2))
    keep = rp.detach() >= 1e-12
    if exclude_inside:
        keep = keep & (rp.detach() >= R.detach()[:, None])
    rps = torch.where(keep, rp, torch.ones_like(rp))
    x = (eN[:, None, :] * d).sum(2)
    c1 = 1.0 - 3.0 * R[:, None] / (4.0 * rps)
    c2 = 3.0 * R[:, None] * x / (4.0 * rps * rps * rps)
    a = c1[:, :, None] * eN[:, None, :] - c2[:, :, None] * d
    a = torch.where(keep[:, :, None], a, torch.zeros_like(a))
    num = (w * a).sum((1, 2))
    den = (a * a).sum((1, 2))
    ok = alive & (den.detach() != 0.0)
    U = torch.where(ok, num / torch.where(ok, den, torch.ones_like(den)), torch.zeros_like(num))
    return gamma[:, None] * U[:, None] * eN


def run(fhat0, r0, V0, M, gamma, R, tau, steps, kT=0.0, seed=0, mode=STOKESLET,
        exclude_inside=False, Fext=None, pinned=None, step0=0):
    """Run `steps` time steps from (fhat0 [15, nz, ny, nx], r0 [n, 3], V0 [n, 3]).

    M, gamma, R: [n] tensors; tau: scalar tensor.  Returns (V_traj, r_traj,
    fhat) with V_traj[t] = V^{t+1} and r_traj[t] = r^{t+1} ([steps, n, 3]) and
    the final post-collision populations.  Every input may require grad.
    """
    nz, ny, nx = fhat0.shape[1:]
    L = torch.tensor([nx, ny, nz], dtype=torch.float64)
    n = r0.shape[0]
    Fx = torch.zeros((n, 3), dtype=torch.float64) if Fext is None else torch.as_tensor(Fext, dtype=torch.float64)
    pin = torch.zeros(n, dtype=torch.bool) if pinned is None else torch.as_tensor(pinned, dtype=torch.bool)
    fhat, r, V = fhat0, r0, V0
    Vs, rs = [], []
    for t in range(steps):
        step = step0 + t
        f = stream(fhat)
        rho, u = moments(f)
        F = torch.zeros((3, nz * ny * nx), dtype=torch.float64)
        if n:
            base = torch.floor(r.detach())
            frac = r - base                                    # [n, 3]
            c = CORNERS[None]                                  # [1, 8, 3]
            d = c - frac[:, None, :]                           # [n, 8, 3]
            fw = torch.where(c > 0, frac[:, None, :], 1.0 - frac[:, None, :])
            Wp = fw.prod(2)                                    # [n, 8]
            idx = (base[:, None, :] + c).long()
            ix = idx[..., 0] % nx
            iy = idx[..., 1] % ny
            iz = idx[..., 2] % nz
            uN = u[:, iz, iy, ix].permute(1, 2, 0)             # [n, 8, 3]
            if mode == STOKESLET:
                FH = stokeslet_force(d, uN, V, R, gamma, exclude_inside)
            elif mode == POINTWISE:
                ur = (Wp[:, :, None] * uN).sum(1)
                FH = -gamma[:, None] * (V - ur)
            else:
                FH = -gamma[:, None] * V
            if kT > 0.0:
                xi = torch.tensor(np.array([noise_xi(seed, step, i) for i in range(n)]),
                                  dtype=torch.float64)
                FR = torch.sqrt(2.0 * gamma * kT)[:, None] * xi
            else:
                FR = torch.zeros((n, 3), dtype=torch.float64)
            if mode != BROWNIAN:
                lin = ((iz * ny + iy) * nx + ix).reshape(-1)
                share = (-FH[:, None, :] * Wp[:, :, None]).reshape(-1, 3)
                F = F.index_add(1, lin, share.t())
            Vn = V + (FH + FR + Fx) / M[:, None]
            rn = r + Vn
            rn = torch.where(rn < 0.0, rn + L, rn)
            rn = torch.where(rn >= L, rn - L, rn)
            V = torch.where(pin[:, None], V, Vn)
            r = torch.where(pin[:, None], r, rn)
        fhat = collide(f, rho, u, F.reshape(3, nz, ny, nx), tau)
        Vs.append(V)
        rs.append(r)
    if steps == 0:
        return (torch.zeros((0, n, 3), dtype=torch.float64),) * 2 + (fhat,)
    return torch.stack(Vs), torch.stack(rs), fhat


def stokes_radius(gamma, tau, rho0=1.0):
    """R with gamma = 6 pi rho0 nu R, nu = (tau - 1/2)/3 (Stokes' law with Eq. 16)."""
    return gamma / (6.0 * math.pi * rho0 * (tau - 0.5) / 3.0)
