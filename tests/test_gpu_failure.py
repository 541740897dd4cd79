"""Failure detection, the conservation budget and checkpoint/resume on the GPU.

Failures are made without faulting the GPU: a NaN or infinity written into one
population through lbp_set_populations, and a bounded device-side wait on a
barrier that nothing completes (lbp_set_wait_probe).  The library must report
each through lbp_check and leave the device usable.
"""
import numpy as np
import pytest

import oracle
from paper_1909_13412_gb300 import lbp
from paper_1909_13412_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, W = oracle.d3q15()
W4 = W[:, None, None, None]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1909_13412_gb300 import build as lbp_build
    lbp_build.build()
    lbp.load()
    torch.cuda.set_device(0)


SHAPE = (10, 12, 16)  # (nz, ny, nx): nx a multiple of 8, so every kernel shape applies


def _handle(prec=lbp.LBP_F32, n=0, kT=1e-4, seed=5, tau=0.8):
    nz, ny, nx = SHAPE
    h = lbp.lbp_create(nx, ny, nz, tau, precision=prec)
    ps = None
    if n:
        ps = wl.uniform_particles(n, SHAPE, 8.0, 0.5, wl.stokes_radius(0.5, tau), kT, 3, 4)
        # away from the corner where the tests below plant a NaN
        ps.r[:] = 6.0 + np.mod(ps.r, 4.0)
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=seed)
    return h, ps


@pytest.mark.parametrize("prec,variant,rows,n", [
    (lbp.LBP_F32, 0, 1, 0), (lbp.LBP_F32, 0, 2, 4), (lbp.LBP_F32, 2, 1, 4),
    (lbp.LBP_BF16, 3, 1, 4), (lbp.LBP_F16, 3, 1, 0), (lbp.LBP_F16, 1, 2, 4), (lbp.LBP_BF16, 0, 2, 0)])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_population_is_reported(prec, variant, rows, n, bad):
    """A non-finite value in one population of one node (injected on the host)
    is caught by the lattice kernel of every shape in the step it is pulled,
    with or without particles (the particles sit away from it), and reported
    once as LBP_ENAN."""
    h, _ = _handle(prec, n)
    lbp.lbp_set_block_shape(h, rows, variant)
    f = np.broadcast_to(W4, (15,) + SHAPE).copy()
    f[7, 1, 2, 3] = bad
    lbp.lbp_set_populations(h, f)
    lbp.lbp_step(h, 1)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_check(h)
    assert ei.value.status == lbp.LBP_ENAN
    assert "lattice" in lbp.lbp_last_error()
    lbp.lbp_check(h)  # reported once, then cleared
    lbp.lbp_destroy(h)


def test_finite_run_reports_nothing():
    h, _ = _handle(lbp.LBP_BF16, 6)
    lbp.lbp_step(h, 20)
    lbp.lbp_check(h)
    lbp.lbp_destroy(h)


@pytest.mark.parametrize("graphs", [True, False])
def test_budget_momentum_and_mass(graphs):
    """Streaming and BGK conserve mass and momentum and the fluid receives
    exactly -F_H (Eqs. 9, 15, 17-20): fluid + particle momentum changes only by
    what F_R + F_ext put into the particles, which lbp_budget tracks on the
    device.  Checked against host sums of the read populations and particles
    and of the read F_R of every step."""
    h, ps = _handle(lbp.LBP_F32, 12)
    lbp.lbp_set_use_graphs(h, graphs)
    g = np.random.default_rng(2)
    fext = 1e-5 * g.standard_normal((12, 3))
    lbp.lbp_particles_set_external_force(h, fext)
    lbp.lbp_step(h, 3)
    lbp.lbp_budget_track(h, True)
    b0 = lbp.lbp_budget(h)
    assert np.all(b0[7:] == 0)
    inj = np.zeros(3)
    fr = np.empty((12, 3))
    for _ in range(25):
        lbp.lbp_step(h, 1)
        lbp.lbp_particles_read(h, f_r=fr)
        inj += (fr + fext).sum(0)
    b1 = lbp.lbp_budget(h)
    assert np.allclose(b1[7:], inj, rtol=1e-12, atol=1e-18)
    P0, P1 = b0[1:4] + b0[4:7] - b0[7:], b1[1:4] + b1[4:7] - b1[7:]
    f = np.empty((15,) + SHAPE)
    lbp.lbp_read_populations(h, f)
    # the fluid keeps its momentum and mass only up to the FP32 rounding of every
    # collided deviation: at most one unit in the last place of each stored value
    # per step (here ~1e-7 out of a total momentum of ~0.15)
    fp32_bound = 25 * 2.0 ** -23 * np.abs(f - W4).sum()
    assert np.all(np.abs(P1 - P0) <= fp32_bound)
    assert abs(b1[0] - b0[0]) <= fp32_bound
    v = np.empty((12, 3))
    lbp.lbp_particles_read(h, v=v)
    assert b1[0] == pytest.approx(f.sum(), rel=1e-13)
    assert np.allclose(b1[1:4], E.T.astype(float) @ f.reshape(15, -1).sum(1), rtol=0, atol=1e-13)
    assert np.allclose(b1[4:7], (ps.M[:, None] * v).sum(0), rtol=1e-14, atol=0)
    lbp.lbp_budget_track(h, False)
    assert np.all(lbp.lbp_budget(h)[7:] == 0)
    lbp.lbp_destroy(h)


def test_staged_kernel_wait_that_runs_out_is_reported_and_recoverable():
    """The bulk-copy staged lattice kernel bounds every mbarrier wait.  With the
    probe on, its consumers wait on a barrier that nothing completes, bounded by
    2^20 cycles (~0.5 ms): lbp_check reports LBP_ETIMEOUT, and after the probe is
    off and a checkpoint is loaded the handle steps on bitwise like a handle that
    never timed out (the kernel drained the copies it had issued before leaving,
    and the force records were reset)."""
    h, _ = _handle(lbp.LBP_F32, 5)
    ref, _ = _handle(lbp.LBP_F32, 5)
    lbp.lbp_set_block_shape(h, 1, 2)
    lbp.lbp_step(h, 3)
    lbp.lbp_step(ref, 3)
    ck = lbp.lbp_checkpoint_save(h)
    lbp.lbp_set_wait_bound(h, 1 << 20)
    lbp.lbp_set_wait_probe(h, True)
    lbp.lbp_step(h, 1)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_check(h)
    assert ei.value.status == lbp.LBP_ETIMEOUT
    lbp.lbp_set_wait_probe(h, False)
    lbp.lbp_set_wait_bound(h, 0)
    lbp.lbp_checkpoint_load(h, ck)
    lbp.lbp_step(h, 4)
    lbp.lbp_step(ref, 4)
    lbp.lbp_check(h)
    lbp.lbp_check(ref)
    fa, fb = np.empty((15,) + SHAPE), np.empty((15,) + SHAPE)
    lbp.lbp_read_populations(h, fa)
    lbp.lbp_read_populations(ref, fb)
    assert np.array_equal(fa, fb)
    va, vb = np.empty((5, 3)), np.empty((5, 3))
    lbp.lbp_particles_read(h, v=va)
    lbp.lbp_particles_read(ref, v=vb)
    assert np.array_equal(va, vb)
    lbp.lbp_destroy(h)
    lbp.lbp_destroy(ref)


@pytest.mark.parametrize("prec", [lbp.LBP_F32, lbp.LBP_BF16, lbp.LBP_F16])
@pytest.mark.parametrize("on_device", [False, True])
def test_checkpoint_resume_is_bitwise(prec, on_device):
    """Save after 40 steps, destroy the handle, recreate it with the same
    configuration, load, continue 50 steps: populations, positions, velocities
    and F_R are bitwise those of an uninterrupted 90-step run (the Philox
    counter of Eqs. 4-5 is the step index, which the checkpoint carries)."""
    def make():
        h, ps = _handle(prec, 9, kT=1e-4, seed=11)
        lbp.lbp_particles_set_external_force(h, np.full((9, 3), 2e-6))
        return h

    full = make()
    lbp.lbp_step(full, 90)
    part = make()
    lbp.lbp_step(part, 40)
    nbytes = lbp.lbp_checkpoint_size(part)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda") if on_device else None
    buf = lbp.lbp_checkpoint_save(part, buf)
    lbp.lbp_destroy(part)
    resumed = make()
    lbp.lbp_checkpoint_load(resumed, buf)
    assert lbp.lbp_get_step_index(resumed) == 40
    lbp.lbp_step(resumed, 50)
    outs = []
    for h in (full, resumed):
        f = np.empty((15,) + SHAPE)
        lbp.lbp_read_populations(h, f)
        r, v, fh, fr = (np.empty((9, 3)) for _ in range(4))
        lbp.lbp_particles_read(h, r, v, fh, fr)
        outs.append((f, r, v, fh, fr))
        lbp.lbp_check(h)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    # a checkpoint of other boxes is refused and changes nothing
    other = lbp.lbp_create(8, 8, 8, 0.8, precision=prec)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_checkpoint_load(other, buf)
    assert ei.value.status == lbp.LBP_EINVAL
    lbp.lbp_destroy(other)
    lbp.lbp_destroy(full)
    lbp.lbp_destroy(resumed)
