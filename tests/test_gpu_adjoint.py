"""The CUDA adjoint (lbp_adjoint_record / lbp_adjoint_backward and the
torch.autograd.Function over them) against independent gradients.

  * FP64 reference gradient (oracle/grad_ref.py: autograd through a PyTorch
    FP64 restatement of the step, itself pinned to the C oracle and to its
    finite differences): every gradient -- tau, kT, gamma_i, R_i, M_i, V0, r0
    and the initial populations -- of a linear functional of both
    trajectories, in all three coupling modes, with noise, an external force
    and a pinned particle; and of a VACF loss.  Tolerance: 1e-4 of the largest
    entry of each gradient (the forward run and the lattice adjoint are FP32).
  * Central finite differences of the C oracle at the 64^3 / 8-particle /
    2000-step relaxation run (checkpoint every 100 steps): dL/dtau,
    dL/dgamma and two components of dL/dV0 of the velocity-relaxation loss,
    to 1e-4 relative.
  * With FP16 or BF16 storage: the same reference, within bounds set by the
    storage's rounding (2^-11 and 2^-8 of the stored deviations).
  * Bitwise: the gradients do not depend on the checkpoint interval and are
    the same on a second run; the backward pass leaves the handle's state
    unchanged; a changed handle is refused.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import grad_ref
from paper_1909_13412_gb300 import adjoint, lbp
from paper_1909_13412_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, W = oracle.d3q15()
SHAPE = (10, 12, 14)  # nz, ny, nx
NAMES = ("tau", "kT", "gamma", "radius", "mass", "v0", "r0", "f0")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1909_13412_gb300 import build as lbp_build
    lbp_build.build()
    lbp.load()
    torch.cuda.set_device(0)


def case(n=5, seed=0):
    g = np.random.default_rng(seed)
    nz, ny, nx = SHAPE
    fhat = W[:, None, None, None] * (1.0 + 0.02 * g.uniform(-1, 1, (15,) + SHAPE))
    r = np.floor(g.uniform(0, 1, (n, 3)) * [nx, ny, nz]) + g.uniform(0.3, 0.7, (n, 3))
    V = g.normal(0, 0.01, (n, 3))
    M = g.uniform(4.0, 8.0, n)
    gamma = g.uniform(0.3, 0.7, n)
    R = g.uniform(0.15, 0.4, n)
    Fext = g.normal(0, 1e-4, (n, 3))
    return dict(fhat=fhat, r=r, V=V, M=M, gamma=gamma, R=R, Fext=Fext)


def leaves(c, tau, kT, device="cpu"):
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device=device, requires_grad=True)
    return dict(tau=t(tau), kT=t(kT), gamma=t(c["gamma"]), radius=t(c["R"]), mass=t(c["M"]),
                v0=t(c["V"]), r0=t(c["r"]), f0=t(c["fhat"]))


def reference(c, tau, kT, steps, seed, mode, exclude, pinned, loss_fn):
    x = leaves(c, tau, kT)
    Vt, rt, _ = grad_ref.run(x["f0"], x["r0"], x["v0"], x["mass"], x["gamma"], x["radius"], x["tau"],
                             steps, kT=x["kT"], seed=seed, mode=mode, exclude_inside=exclude,
                             Fext=c["Fext"], pinned=pinned)
    loss_fn(Vt, rt).backward()
    return {k: (v.grad.numpy() if v.grad is not None else np.zeros(v.shape)) for k, v in x.items()}, Vt.detach().numpy()


def gpu(c, tau, kT, steps, seed, mode, exclude, pinned, loss_fn, C, precision=lbp.LBP_F32):
    nz, ny, nx = SHAPE
    x = leaves(c, tau, kT)
    spec = adjoint.RunSpec(nx, ny, nz, steps, C, seed, mode, int(exclude), precision)
    pin = None if pinned is None else torch.tensor(pinned)
    Vt, rt = adjoint.trajectory(x["tau"], x["gamma"], x["radius"], x["mass"], x["v0"], x["r0"], spec,
                                kT=x["kT"], f0=x["f0"], f_ext=torch.tensor(c["Fext"]), pinned=pin)
    loss_fn(Vt, rt).backward()
    return {k: (v.grad.numpy() if v.grad is not None else np.zeros(v.shape)) for k, v in x.items()}, Vt.detach().cpu().numpy()


def linear_loss(steps, n, seed=9):
    g = np.random.default_rng(seed)
    cV = g.normal(0, 1, (steps, n, 3))
    cr = g.normal(0, 1, (steps, n, 3))

    def f(Vt, rt):
        return (torch.tensor(cV, device=Vt.device) * Vt).sum() + (torch.tensor(cr, device=rt.device) * rt).sum()
    return f


def assert_close(got, want, rtol, names=NAMES):
    for k in names:
        scale = np.max(np.abs(want[k]))
        err = np.max(np.abs(got[k] - want[k]))
        assert err <= rtol * max(scale, 1e-300) or (scale == 0 and err == 0), (k, err, scale)


MODES = [(lbp.LBP_STOKESLET, 0, 1e-4), (lbp.LBP_STOKESLET, 1, 0.0),
         (lbp.LBP_POINTWISE, 0, 1e-4), (lbp.LBP_BROWNIAN, 0, 1e-4)]


@pytest.mark.parametrize("mode,exclude,kT", MODES)
def test_adjoint_matches_fp64_reference(mode, exclude, kT):
    c = case()
    steps = 40
    pinned = np.array([0, 0, 0, 1, 0], np.uint8)
    loss = linear_loss(steps, 5)
    want, Vw = reference(c, 0.8, kT, steps, 11, mode, exclude, pinned, loss)
    got, Vg = gpu(c, 0.8, kT, steps, 11, mode, exclude, pinned, loss, C=7)
    # the forward trajectories agree to FP32 accuracy
    assert np.max(np.abs(Vg - Vw)) <= 1e-5 * np.max(np.abs(Vw))
    names = [k for k in NAMES if not (k == "kT" and kT == 0.0)]
    if mode == lbp.LBP_BROWNIAN:
        names = [k for k in names if k not in ("tau", "f0", "radius")]
        assert np.all(got["tau"] == 0) and np.all(got["f0"] == 0)
    if mode == lbp.LBP_POINTWISE:
        names = [k for k in names if k != "radius"]
    assert_close(got, want, 1e-4, names)


# forward-trajectory and gradient bounds (relative to the largest entry) for
# 2-byte storage: FP16 rounds the scaled deviations to 2^-11, BF16 the
# deviations to 2^-8; measured on GB300 (40 steps): FP16 forward 5e-6,
# gradients <= 1.4e-4 (tau; the rest <= 2e-5); BF16 forward 3.7e-5, gradients
# <= 2.8e-4 (tau; the rest <= 8e-5)
TWO_BYTE_BOUNDS = {lbp.LBP_F16: (5e-5, 1e-3), lbp.LBP_BF16: (3e-4, 2e-3)}


@pytest.mark.parametrize("prec", [lbp.LBP_F16, lbp.LBP_BF16])
def test_adjoint_with_two_byte_storage(prec):
    """The adjoint of a run whose populations are stored as FP16 or BF16
    deviations: the recording and the reverse sweep use the handle's storage
    (the replayed forward steps round exactly as the recorded ones) and the
    lattice adjoint reads the rounded populations.  Against the FP64 reference
    of the unrounded method the trajectories and every gradient carry the
    storage's rounding, within the bounds above."""
    c = case(seed=7)
    steps = 40
    loss = linear_loss(steps, 5, seed=2)
    want, Vw = reference(c, 0.8, 1e-4, steps, 11, lbp.LBP_STOKESLET, 0, None, loss)
    got, Vg = gpu(c, 0.8, 1e-4, steps, 11, lbp.LBP_STOKESLET, 0, None, loss, C=7, precision=prec)
    fwd_tol, grad_tol = TWO_BYTE_BOUNDS[prec]
    assert np.max(np.abs(Vg - Vw)) <= fwd_tol * np.max(np.abs(Vw))
    assert_close(got, want, grad_tol)


def test_adjoint_of_a_vacf_loss():
    c = case(n=6, seed=3)
    steps, K = 60, 12

    def loss(Vt, rt):
        C_k = adjoint.vacf(Vt, K)
        return ((C_k / C_k[0].detach() - torch.linspace(1.0, 0.5, K + 1, dtype=torch.float64,
                                                          device=Vt.device)) ** 2).sum()
    want, _ = reference(c, 0.7, 2e-4, steps, 4, lbp.LBP_STOKESLET, 0, None, loss)
    got, _ = gpu(c, 0.7, 2e-4, steps, 4, lbp.LBP_STOKESLET, 0, None, loss, C=16)
    assert_close(got, want, 1e-4)


BATCH = [((14, 12, 10), 0.6, 4), ((9, 8, 12), 0.8, 0), ((16, 6, 5), 1.0, 3)]  # (nx, ny, nz), tau, particles


def _box_leaves(b, shape, tau, n):
    nx, ny, nz = shape
    g = np.random.default_rng(70 + b)
    fhat = W[:, None, None, None] * (1.0 + 0.02 * g.uniform(-1, 1, (15, nz, ny, nx)))
    r = np.floor(g.uniform(0, 1, (n, 3)) * [nx, ny, nz]) + g.uniform(0.3, 0.7, (n, 3))
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True)
    return dict(tau=t(tau), gamma=t(g.uniform(0.3, 0.7, n)), radius=t(g.uniform(0.15, 0.4, n)),
                mass=t(g.uniform(4.0, 8.0, n)), v0=t(g.normal(0, 0.01, (n, 3))), r0=t(r), f0=t(fhat))


def test_batched_autograd_run_equals_its_boxes():
    """batch_trajectory over three boxes of different sizes and relaxation times
    (one without particles) under a loss that mixes them -- the ensemble VACF
    of Section 3 over all particles plus a linear functional: the trajectories
    and every gradient (tau per box, gamma, R, M, V0, r0, f0) equal, bit for bit,
    those of each box run alone through trajectory() and driven back with its
    slice of the same upstream gradient; the particle-free box gets zero."""
    steps, C, K = 25, 10, 8
    per = [_box_leaves(b, *bx) for b, bx in enumerate(BATCH)]
    counts = tuple(n for _, _, n in BATCH)
    cat = lambda k: torch.cat([p[k].detach() for p in per if p[k].numel()], 0)
    bl = {k: cat(k).clone().requires_grad_(True) for k in ("gamma", "radius", "mass", "v0", "r0")}
    bl["tau"] = torch.tensor([tau for _, tau, _ in BATCH], dtype=torch.float64, requires_grad=True)
    bl["f0"] = torch.cat([p["f0"].detach().reshape(15, -1) for p in per], 1).requires_grad_(True)
    spec = adjoint.BatchSpec(tuple(s for s, _, _ in BATCH), counts, steps, C)
    Vt, rt = adjoint.batch_trajectory(bl["tau"], bl["gamma"], bl["radius"], bl["mass"], bl["v0"],
                                      bl["r0"], spec, f0=bl["f0"])
    n = sum(counts)
    Vd, rd = Vt.detach().requires_grad_(True), rt.detach().requires_grad_(True)
    C_k = adjoint.vacf(Vd, K)
    loss = ((C_k / C_k[0].detach() - 0.5) ** 2).sum() + linear_loss(steps, n, seed=4)(Vd, rd)
    gV, gR = torch.autograd.grad(loss, (Vd, rd))
    torch.autograd.backward((Vt, rt), (gV, gR))
    p0, node0 = 0, 0
    for b, ((nx, ny, nz), tau, nb) in enumerate(BATCH):
        Nb = nx * ny * nz
        x = per[b]
        if nb == 0:
            assert bl["tau"].grad[b].item() == 0.0
            assert not torch.any(bl["f0"].grad[:, node0:node0 + Nb])
        else:
            sl = slice(p0, p0 + nb)
            Vb, rb = adjoint.trajectory(x["tau"], x["gamma"], x["radius"], x["mass"], x["v0"], x["r0"],
                                        adjoint.RunSpec(nx, ny, nz, steps, C), f0=x["f0"])
            assert torch.equal(Vb, Vt[:, sl].detach()) and torch.equal(rb, rt[:, sl].detach()), b
            torch.autograd.backward((Vb, rb), (gV[:, sl].contiguous(), gR[:, sl].contiguous()))
            assert x["tau"].grad.item() == bl["tau"].grad[b].item() != 0.0, b
            for k in ("gamma", "radius", "mass", "v0", "r0"):
                assert torch.equal(x[k].grad, bl[k].grad[sl]), (b, k)
            assert torch.equal(x["f0"].grad.reshape(15, -1), bl["f0"].grad[:, node0:node0 + Nb]), b
        p0 += nb
        node0 += Nb


def test_checkpoint_interval_and_repeat_are_bitwise_invariant():
    c = case(seed=5)
    steps = 30
    loss = linear_loss(steps, 5, seed=2)
    runs = [gpu(c, 0.9, 1e-4, steps, 8, lbp.LBP_STOKESLET, 0, None, loss, C=C)[0] for C in (1, 7, 30, 7)]
    for other in runs[1:]:
        for k in NAMES:
            assert np.array_equal(other[k], runs[0][k]), k


def test_backward_leaves_the_handle_and_refuses_changes():
    c = case(seed=6)
    nz, ny, nx = SHAPE

    def make():
        h = lbp.lbp_create(nx, ny, nz, 0.8)
        lbp.lbp_set_populations(h, c["fhat"])
        lbp.lbp_particles_add(h, c["r"], c["V"], c["M"], c["gamma"], c["R"])
        lbp.lbp_particles_set_params(h, kT=1e-4, seed=1)
        lbp.lbp_vacf_configure(h, 8)
        return h
    h1, h2 = make(), make()
    n = 5
    for h in (h1, h2):
        lbp.lbp_adjoint_record(h, 20, 6)
    g = np.random.default_rng(0).normal(0, 1, (20, n, 3))
    out = {"tau": np.zeros(1), "v0": np.zeros((n, 3)), "f0": np.zeros((15, h1.N))}
    lbp.lbp_adjoint_backward(h1, 20, g, None, out)
    assert np.all(np.isfinite(out["f0"])) and out["tau"][0] != 0.0
    assert lbp.lbp_get_step_index(h1) == 20
    for h in (h1, h2):
        lbp.lbp_step(h, 70)
    f1, f2 = np.empty((15, h1.N)), np.empty((15, h1.N))
    lbp.lbp_read_populations(h1, f1)
    lbp.lbp_read_populations(h2, f2)
    assert np.array_equal(f1, f2)
    p1 = [np.empty((n, 3)) for _ in range(4)]
    p2 = [np.empty((n, 3)) for _ in range(4)]
    lbp.lbp_particles_read(h1, *p1)
    lbp.lbp_particles_read(h2, *p2)
    for a, b in zip(p1, p2):
        assert np.array_equal(a, b)
    cs1, cs2 = np.empty(9), np.empty(9)
    ct = np.empty(9, np.int64)
    lbp.lbp_vacf_read(h1, cs1, ct)
    lbp.lbp_vacf_read(h2, cs2, ct)
    assert np.array_equal(cs1, cs2)
    # the handle moved on: the recording no longer matches it
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_adjoint_backward(h1, 20, g, None, {"tau": np.zeros(1)})
    assert ei.value.status == lbp.LBP_ESTATE
    lbp.lbp_adjoint_record(h2, 5, 2)
    lbp.lbp_particles_set_state(h2, v=np.zeros((n, 3)))
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_adjoint_backward(h2, 5, None, None, {"tau": np.zeros(1)})
    assert ei.value.status == lbp.LBP_ESTATE
    lbp.lbp_destroy(h1)
    lbp.lbp_destroy(h2)


def test_relaxation_run_64_against_oracle_finite_differences():
    """64^3, 8 kicked particles, 2000 steps, checkpoint every 100 steps; loss =
    mean squared deviation of V_i(t) from V_i(0) exp(-t gamma / M)."""
    w = wl.ADJOINT_64
    ps = wl.kicked_particles(w)
    nz, ny, nx = w.shape_zyx
    steps, C = w.steps, w.extra["checkpoint_every"]
    t_relax = w.M / w.gamma
    tgrid = np.arange(1, steps + 1)
    target = ps.V[None] * np.exp(-tgrid / t_relax)[:, None, None]

    def J_numpy(Vt):
        return float(np.mean((Vt - target) ** 2))

    tau_t = torch.tensor(w.tau, dtype=torch.float64, requires_grad=True)
    gam_t = torch.tensor(w.gamma, dtype=torch.float64, requires_grad=True)
    v0_t = torch.tensor(ps.V, requires_grad=True)
    n = ps.n
    spec = adjoint.RunSpec(nx, ny, nz, steps, C)
    Vt, _ = adjoint.trajectory(tau_t, gam_t.expand(n).contiguous(), torch.tensor(ps.R), torch.tensor(ps.M),
                               v0_t, torch.tensor(ps.r), spec)
    loss = torch.mean((Vt - torch.tensor(target, device=Vt.device)) ** 2)
    loss.backward()
    got = {"tau": float(tau_t.grad), "gamma": float(gam_t.grad), "v0_00": float(v0_t.grad[0, 0]),
           "v0_31": float(v0_t.grad[3, 1])}

    def J_oracle(tau=w.tau, gamma=w.gamma, V=ps.V):
        o = oracle.Sim(nx, ny, nz, tau)
        o.add_particles(ps.r, V, ps.M, np.full(n, gamma), ps.R)
        Vs = np.empty((steps, n, 3))
        for t in range(steps):
            o.step(1)
            Vs[t] = o.particles()[1]
        o.close()
        return J_numpy(Vs)

    def dV(i, k, h):
        Vp, Vm = ps.V.copy(), ps.V.copy()
        Vp[i, k] += h
        Vm[i, k] -= h
        return (J_oracle(V=Vp) - J_oracle(V=Vm)) / (2 * h)

    want = {"tau": (J_oracle(tau=w.tau + 1e-4) - J_oracle(tau=w.tau - 1e-4)) / 2e-4,
            "gamma": (J_oracle(gamma=w.gamma + 1e-4) - J_oracle(gamma=w.gamma - 1e-4)) / 2e-4,
            "v0_00": dV(0, 0, 1e-6), "v0_31": dV(3, 1, 1e-6)}
    for k in want:
        assert abs(got[k] - want[k]) <= 1e-4 * abs(want[k]), (k, got[k], want[k])
