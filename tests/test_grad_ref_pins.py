"""Pins of the FP64 reference gradient (oracle/grad_ref.py), CPU only.

The reference gradient is autograd through a PyTorch FP64 restatement of the
time step.  Two independent checks hold it to the paper's method:

  * its forward run equals the C oracle (lbp_oracle.c) step by step: particle
    velocities and positions after every step and the final populations, to
    1e-12 relative, in all three coupling modes, with noise, an external force
    and a pinned particle;
  * its gradient of a linear functional of the trajectories equals the central
    finite difference of the C oracle run with respect to tau, gamma_i, R_i,
    M_i, V0, r0 and single initial populations, to 1e-6 relative (steps h are
    chosen per parameter so that truncation and rounding stay below 1e-8).
"""
import numpy as np
import pytest

import oracle
from oracle import grad_ref

torch = pytest.importorskip("torch")

E, W = oracle.d3q15()
SHAPE = (9, 10, 12)  # nz, ny, nx


def case(n=4, seed=0):
    g = np.random.default_rng(seed)
    nz, ny, nx = SHAPE
    fhat = W[:, None, None, None] * (1.0 + 0.02 * g.uniform(-1, 1, (15,) + SHAPE))
    # positions away from cell faces so that no particle changes cell under a
    # finite-difference step
    r = np.floor(g.uniform(0, 1, (n, 3)) * [nx, ny, nz]) + g.uniform(0.25, 0.75, (n, 3))
    V = g.normal(0, 0.01, (n, 3))
    M = g.uniform(4.0, 8.0, n)
    gamma = g.uniform(0.3, 0.7, n)
    R = g.uniform(0.15, 0.4, n)
    Fext = g.normal(0, 1e-4, (n, 3))
    return fhat, r, V, M, gamma, R, Fext


def run_oracle(fhat, r, V, M, gamma, R, tau, steps, kT, seed, mode, exclude, Fext, pinned):
    nz, ny, nx = SHAPE
    o = oracle.Sim(nx, ny, nz, tau)
    o.set_fhat(fhat)
    o.add_particles(r, V, M, gamma, R)
    o.set_params(kT=kT, seed=seed, mode=mode, exclude_inside=exclude)
    o.set_external(Fext, pinned)
    Vs, rs = [], []
    for _ in range(steps):
        o.step(1)
        rr, VV, _, _ = o.particles()
        Vs.append(VV)
        rs.append(rr)
    out = np.array(Vs), np.array(rs), o.fhat()
    o.close()
    return out


def run_ref(fhat, r, V, M, gamma, R, tau, steps, kT, seed, mode, exclude, Fext, pinned, grad=False):
    t = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=grad)
    args = [t(fhat), t(r), t(V), t(M), t(gamma), t(R), t(tau)]
    Vt, rt, fh = grad_ref.run(*args, steps, kT=kT, seed=seed, mode=mode, exclude_inside=exclude,
                              Fext=Fext, pinned=pinned)
    return args, Vt, rt, fh


MODES = [(oracle.STOKESLET, False, 1e-4), (oracle.STOKESLET, True, 0.0),
         (oracle.POINTWISE, False, 1e-4), (oracle.BROWNIAN, False, 1e-4)]


@pytest.mark.parametrize("mode,exclude,kT", MODES)
def test_reference_forward_equals_c_oracle(mode, exclude, kT):
    fhat, r, V, M, gamma, R, Fext = case()
    pinned = np.array([0, 0, 1, 0], np.uint8)
    steps = 25
    Vo, ro, fo = run_oracle(fhat, r, V, M, gamma, R, 0.8, steps, kT, 7, mode, exclude, Fext, pinned)
    _, Vt, rt, fh = run_ref(fhat, r, V, M, gamma, R, 0.8, steps, kT, 7, mode, exclude, Fext, pinned)
    sv = np.max(np.abs(Vo))
    assert np.max(np.abs(Vt.numpy() - Vo)) <= 1e-12 * sv
    assert np.max(np.abs(rt.numpy() - ro)) <= 1e-12 * SHAPE[2]
    dev = np.max(np.abs(fo - W[:, None, None, None]))
    assert np.max(np.abs(fh.detach().numpy() - fo)) <= 1e-12 * dev
    # the fluid did move and the particles did interact with it
    assert dev > 1e-5 and np.max(np.abs(Vo[-1] - V)) > 1e-5


@pytest.mark.parametrize("mode,exclude,kT", MODES)
def test_reference_gradient_equals_oracle_finite_differences(mode, exclude, kT):
    fhat, r, V, M, gamma, R, Fext = case(seed=1)
    pinned = np.zeros(4, np.uint8)
    tau, steps, seed = 0.8, 12, 3
    g = np.random.default_rng(5)
    cV = g.normal(0, 1, (steps, 4, 3))
    cr = g.normal(0, 1, (steps, 4, 3))

    def J(Vt, rt):
        return float(np.sum(cV * Vt) + np.sum(cr * rt))

    args, Vt, rt, _ = run_ref(fhat, r, V, M, gamma, R, tau, steps, kT, seed, mode, exclude, Fext,
                              pinned, grad=True)
    loss = (torch.tensor(cV) * Vt).sum() + (torch.tensor(cr) * rt).sum()
    loss.backward()
    # an input the loss does not depend on (tau and fhat in the uncoupled Eq. 6
    # mode) gets no gradient from autograd: zero
    gf, gr, gV, gM, gg, gR, gt = (a.grad.numpy() if a.grad is not None else np.zeros(a.shape)
                                  for a in args)

    base = dict(fhat=fhat, r=r, V=V, M=M, gamma=gamma, R=R, tau=tau)

    def fd(name, index, h):
        vals = []
        for sgn in (1.0, -1.0):
            p = {k: (np.array(v, dtype=np.float64) if k != "tau" else v) for k, v in base.items()}
            if name == "tau":
                p["tau"] = tau + sgn * h
            else:
                p[name][index] += sgn * h
            Vo, ro, _ = run_oracle(p["fhat"], p["r"], p["V"], p["M"], p["gamma"], p["R"], p["tau"],
                                   steps, kT, seed, mode, exclude, Fext, pinned)
            vals.append(J(Vo, ro))
        return (vals[0] - vals[1]) / (2 * h)

    checks = [("tau", None, 1e-5, float(gt)),
              ("gamma", 1, 1e-6, gg[1]), ("M", 2, 1e-5, gM[2]),
              ("V", (0, 0), 1e-7, gV[0, 0]), ("V", (3, 2), 1e-7, gV[3, 2]),
              ("r", (1, 1), 1e-6, gr[1, 1]), ("r", (2, 0), 1e-6, gr[2, 0]),
              ("fhat", (7, 4, 5, 6), 1e-6, gf[7, 4, 5, 6]), ("fhat", (0, 1, 2, 3), 1e-6, gf[0, 1, 2, 3])]
    if mode == oracle.STOKESLET:
        checks.append(("R", 0, 1e-6, gR[0]))
    scale = max(abs(c[3]) for c in checks)
    for name, index, h, got in checks:
        want = fd(name, index, h)
        assert abs(got - want) <= 1e-6 * max(abs(want), 1e-3 * scale), (name, index, got, want)
