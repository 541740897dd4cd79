"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written in each test):
  * bit-exact: Philox blocks, the random force F_R, cell indices and trilinear
    weights (integer/bit-level work, same IEEE expressions on both sides);
  * populations after one step: |g_gpu - g_oracle| <= 1e-6 max|f_oracle - w|
    (FP32 storage of the deviation g = f - w carries ~6e-8 relative rounding);
  * particle velocity after 10^3 steps (single kicked particle): 1e-4 relative.
"""
import math
import warnings

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


def gpu_sim(shape_zyx, tau, ps=None, kT=0.0, seed=0, mode=lbp.LBP_STOKESLET, exclude=0, graphs=True):
    nz, ny, nx = shape_zyx
    h = lbp.lbp_create(nx, ny, nz, tau)
    lbp.lbp_set_use_graphs(h, graphs)
    if ps is not None:
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=seed, mode=mode, fit_exclude_inside=exclude)
    return h


def oracle_sim(shape_zyx, tau, ps=None, kT=0.0, seed=0, mode=0, exclude=0):
    nz, ny, nx = shape_zyx
    o = oracle.Sim(nx, ny, nz, tau)
    if ps is not None:
        o.add_particles(ps.r, ps.V, ps.M, ps.gamma, ps.R)
        o.set_params(kT=kT, seed=seed, mode=mode, exclude_inside=exclude)
    return o


def gpu_pops(h):
    f = np.empty((15, h.nz, h.ny, h.nx))
    lbp.lbp_read_populations(h, f)
    return f


def gpu_particles(h):
    n = h.np
    out = [np.empty((n, 3)) for _ in range(4)]
    lbp.lbp_particles_read(h, *out)
    return out


def dev_scale(fo):
    return np.max(np.abs(fo - W4))


# The oracle's own FP64 rounding leaves ~1e-16 absolute noise even in a state
# at rest; comparisons of populations carry this floor.
F64_FLOOR = 1e-14


# ---------------------------------------------------------------- bit-exact pieces
def test_philox_bit_exact():
    g = np.random.default_rng(0)
    n = 4096
    ctr = g.integers(0, 2 ** 63, (n, 4), dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    ctr[:16] = np.arange(64, dtype=np.uint64).reshape(16, 4)
    key = np.array([0x0123456789ABCDEF, 0xFEDCBA9876543210], np.uint64)
    out = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
    lbp.lbp_philox4x64_10(torch.from_numpy(ctr.view(np.int64)).cuda(),
                          torch.from_numpy(key.view(np.int64)).cuda(), out, n)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    for i in list(range(64)) + list(range(n - 64, n)):
        assert np.array_equal(got[i], oracle.philox4x64_10(ctr[i], key)), i


def test_random_force_bit_exact():
    shape = (6, 7, 9)
    ps = wl.uniform_particles(50, shape, 10.0, 0.5, 0.26, 1e-4, 3, 4)
    h = gpu_sim(shape, 0.8, ps, kT=2.5e-4, seed=1234)
    o = oracle_sim(shape, 0.8, ps, kT=2.5e-4, seed=1234)
    for n in range(3):
        lbp.lbp_step(h, 1)
        o.step(1)
        _, _, _, FR = gpu_particles(h)
        _, _, _, FRo = o.particles()
        assert np.array_equal(FR.view(np.uint64), FRo.view(np.uint64)), n
    lbp.lbp_set_step_index(h, 10 ** 12)
    o.set_step(10 ** 12)
    lbp.lbp_step(h, 1)
    o.step(1)
    assert np.array_equal(gpu_particles(h)[3], o.particles()[3])


def test_cell_indexing_bit_exact():
    shape = (12, 11, 10)
    g = np.random.default_rng(5)
    r = g.random((300, 3)) * np.array([10, 11, 12.0])
    r[:6] = [[0, 0, 0], [9.999999999999998, 10.999999999999998, 11.999999999999998],
             [3.0, 4.0, 5.0], [0.5, 0.5, 0.5], [1e-300, 2.0, 7.25], [9.5, 0.1, 11.0]]
    ps = wl.ParticleSet(r, np.zeros_like(r), np.full(300, 10.0), np.full(300, 0.5), np.full(300, 0.2))
    h = gpu_sim(shape, 0.8, ps)
    base = np.empty((300, 3), np.int32)
    frac = np.empty((300, 3))
    lbp.lbp_particles_read_cells(h, base, frac)
    for i in range(300):
        b, d, _ = oracle.corners(r[i])
        assert np.array_equal(base[i], b)
        assert np.array_equal(frac[i], -d[0]), i   # corner 0 offset is -q


def test_reaction_force_shares_are_trilinear_and_exact():
    """A pinned particle at an off-centre position in fluid at rest: after one
    step the momentum the fluid received equals -F_H exactly (fixed-point shares
    sum exactly) and the node-by-node force matches the oracle's trilinear
    spreading to 2^-30 relative."""
    shape = (8, 8, 8)
    r = np.array([[3.3, 4.7, 2.15]])
    ps = wl.ParticleSet(r, np.array([[0.004, -0.003, 0.002]]), np.array([10.0]), np.array([0.5]),
                        np.array([0.26]))
    h = gpu_sim(shape, 0.8, ps)
    lbp.lbp_particles_set_external_force(h, None, np.array([1], np.uint8))
    lbp.lbp_step(h, 1)
    _, _, FH, _ = gpu_particles(h)
    f = gpu_pops(h)
    # from rest, one collision: fhat - w = body-force term 3 w_a F.e_a exactly where F != 0
    G = f - W4
    Fnode = np.einsum("ai,azyx->izyx", E.astype(float), G)
    assert np.allclose(Fnode.reshape(3, -1).sum(1), -FH[0], rtol=1e-6, atol=1e-15)
    o = oracle_sim(shape, 0.8, ps)
    o.set_external(None, np.array([1], np.uint8))
    o.step(1)
    Fo = o.spread_only()
    assert np.allclose(Fnode, Fo, rtol=1e-5, atol=1e-6 * np.abs(FH).max())

# ---------------------------------------------------------------- lattice step
@pytest.mark.parametrize("shape,tau", [((13, 21, 300), 0.8), ((5, 3, 37), 0.6), ((1, 1, 1), 1.3),
                                       ((2, 130, 7), 0.55)])
@pytest.mark.parametrize("graphs", [True, False])
def test_stream_collide_one_step(shape, tau, graphs):
    """Random non-equilibrium state, no particles: several 128-node x-chunks and
    a ragged tail (nx = 300), odd sizes and 1-node boxes."""
    f0 = wl.perturbed_populations(W, shape, 0.05, 17)
    h = gpu_sim(shape, tau, graphs=graphs)
    lbp.lbp_set_populations(h, f0)
    lbp.lbp_step(h, 1)
    o = oracle_sim(shape, tau)
    o.set_fhat(f0)
    o.step(1)
    fo = o.fhat()
    err = np.max(np.abs(gpu_pops(h) - fo))
    assert err <= 1e-6 * dev_scale(fo) + F64_FLOOR, err / dev_scale(fo)


def test_set_read_populations_roundtrip_and_rest_state():
    shape = (4, 5, 6)
    h = gpu_sim(shape, 0.8)
    assert np.array_equal(gpu_pops(h), np.broadcast_to(W4, (15,) + shape))
    f0 = wl.perturbed_populations(W, shape, 0.1, 1)
    lbp.lbp_set_populations(h, f0)
    got = gpu_pops(h)
    # stored as FP32 deviations: |error| <= 2^-24 |f - w|
    assert np.all(np.abs(got - f0) <= 2.0 ** -24 * np.abs(f0 - W4) + 1e-300)


def test_fields_parity_and_device_pointers():
    shape = (9, 10, 11)
    f0 = wl.perturbed_populations(W, shape, 0.05, 4)
    h = gpu_sim(shape, 0.7)
    lbp.lbp_set_populations(h, torch.from_numpy(f0.reshape(-1)).cuda())
    o = oracle_sim(shape, 0.7)
    o.set_fhat(f0)
    rho, u, p = (torch.empty(n * 990, dtype=torch.float64, device="cuda") for n in (1, 3, 1))
    lbp.lbp_read_fields(h, rho, u, p)
    torch.cuda.synchronize()
    ro, uo, po = o.fields()
    scale = dev_scale(f0)
    assert np.max(np.abs(rho.cpu().numpy().reshape(shape) - ro)) <= 1e-6 * scale
    assert np.max(np.abs(u.cpu().numpy().reshape((3,) + shape) - uo)) <= 1e-6 * scale
    assert np.max(np.abs(p.cpu().numpy().reshape(shape) - po)) <= 1e-6 * scale


def test_many_steps_conserve_mass_and_stay_close():
    shape = (16, 16, 16)
    f0 = wl.perturbed_populations(W, shape, 0.02, 9)
    h = gpu_sim(shape, 0.9)
    lbp.lbp_set_populations(h, f0)
    lbp.lbp_step(h, 100)
    o = oracle_sim(shape, 0.9)
    o.set_fhat(f0)
    o.step(100)
    fo = o.fhat()
    f = gpu_pops(h)
    assert abs(f.sum() - f0.sum()) <= 1e-6 * dev_scale(f0) * 15 * 4096
    assert np.max(np.abs(f - fo)) <= 1e-5 * dev_scale(f0) + F64_FLOOR


# ---------------------------------------------------------------- coupled step
def test_kicked_particle_relaxation_1000_steps():
    """The 32^3 single-particle relaxation run: V after 10^3 steps to 1e-4."""
    w = wl.RELAXATION_32
    ps = wl.relaxation_particle(w)
    h = gpu_sim(w.shape_zyx, w.tau, ps)
    o = oracle_sim(w.shape_zyx, w.tau, ps)
    lbp.lbp_step(h, 1)
    o.step(1)
    _, V1, FH1, _ = gpu_particles(h)
    _, V1o, FH1o, _ = o.particles()
    assert FH1[0, 0] / (-0.5 * 0.01) == pytest.approx(1.40724, rel=1e-5)
    # the fit is FP64 on the device and the fluid is exactly at rest at the first
    # step (u^N = 0): only the order of FP64 roundings differs from the oracle
    assert np.allclose(FH1, FH1o, rtol=1e-12, atol=0)
    lbp.lbp_step(h, 999)
    o.step(999)
    r, V, _, _ = gpu_particles(h)
    ro, Vo, _, _ = o.particles()
    assert np.max(np.abs(V - Vo)) <= 1e-4 * np.max(np.abs(Vo))
    assert np.max(np.abs(r - ro)) <= 1e-6
    lbp.lbp_check(h)


@pytest.mark.parametrize("r", [[4.3, 5.6, 3.7], [4.0, 5.0, 3.0]])
def test_pointwise_friction_in_an_affine_flow(r):
    """Eq. 7 on the device: in the affine flow u0 + A x of the oracle's Eq. 7 pin
    (streamed populations at the equilibrium of Eq. 17) the point-wise friction is
    -gamma (V - u0 - A r_i) in closed form; the FP32 deviation storage of the
    populations limits the agreement to ~1e-7 of |u|, i.e. 1e-6 of F_H."""
    from test_oracle_pins import _A, _U0, _linear_flow_populations
    L = 10
    r = np.array(r)
    V, gamma = np.array([0.01, -0.004, 0.006]), 0.45
    h = lbp.lbp_create(L, L, L, 0.8)
    lbp.lbp_set_populations(h, _linear_flow_populations(L, _U0, _A))
    lbp.lbp_particles_add(h, r[None].copy(), V[None].copy(), np.array([10.0]), np.array([gamma]),
                          np.array([0.3]))
    lbp.lbp_particles_set_params(h, mode=lbp.LBP_POINTWISE)
    lbp.lbp_step(h, 1)
    FH = gpu_particles(h)[2][0]
    lbp.lbp_destroy(h)
    expect = -gamma * (V - (_U0 + _A @ r))
    assert np.allclose(FH, expect, rtol=0, atol=1e-6 * np.abs(expect).max())


@pytest.mark.parametrize("mode", [lbp.LBP_STOKESLET, lbp.LBP_POINTWISE, lbp.LBP_BROWNIAN])
@pytest.mark.parametrize("exclude", [0, 1])
def test_coupled_brownian_particles(mode, exclude):
    """40 particles, some sharing cells and nodes, with noise: 60 steps."""
    shape = (14, 17, 19)
    ps = wl.uniform_particles(40, shape, 10.0, 0.5, wl.stokes_radius(0.5, 0.7), 1e-4, 21, 22)
    Lxyz = np.array([19.0, 17.0, 14.0])
    ps.r[1] = np.floor(ps.r[0]) + [0.1, 0.8, 0.45]               # same cell as particle 0
    ps.r[3] = (np.floor(ps.r[2]) + [1.2, 0.3, 0.6]) % Lxyz       # shares four nodes with particle 2
    ps.r[4] = [18.9, 16.95, 13.99]   # touches the periodic seams in x, y and z
    h = gpu_sim(shape, 0.7, ps, kT=1e-4, seed=77, mode=mode, exclude=exclude)
    o = oracle_sim(shape, 0.7, ps, kT=1e-4, seed=77, mode=mode, exclude=exclude)
    lbp.lbp_step(h, 60)
    o.step(60)
    r, V, FH, FR = gpu_particles(h)
    ro, Vo, FHo, FRo = o.particles()
    assert np.array_equal(FR, FRo)
    vs = np.max(np.abs(Vo))
    assert np.max(np.abs(V - Vo)) <= 1e-5 * vs
    assert np.max(np.abs(FH - FHo)) <= 1e-5 * np.max(np.abs(FHo))
    d = np.abs(r - ro)
    d = np.minimum(d, np.array([19, 17, 14.0]) - d)
    assert np.max(d) <= 1e-6
    fo = o.fhat()
    assert np.max(np.abs(gpu_pops(h) - fo)) <= 1e-5 * dev_scale(fo) + F64_FLOOR
    lbp.lbp_check(h)


@pytest.mark.parametrize("device", [False, True])
def test_step_exchange_equals_the_separate_calls(device):
    """lbp_step_exchange(f_ext, r, v) = set_external_force + step + particles_read,
    bitwise, step after step; f_ext = None keeps the previous forces."""
    shape = (12, 13, 14)
    ps = wl.uniform_particles(9, shape, 8.0, 0.5, wl.stokes_radius(0.5, 0.8), 1e-4, 3, 4)
    ha = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=9)
    hb = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=9)
    g = np.random.default_rng(1)
    n = ps.n
    for k in range(6):
        f = None if k == 3 else g.normal(0, 1e-5, (n, 3))
        if f is not None:
            lbp.lbp_particles_set_external_force(ha, f)
        lbp.lbp_step(ha, 1)
        ra, va = np.empty((n, 3)), np.empty((n, 3))
        lbp.lbp_particles_read(ha, r=ra, v=va)
        if device:
            ft = None if f is None else torch.tensor(f, device="cuda")
            rb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            vb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            lbp.lbp_step_exchange(hb, ft, rb, vb)
            torch.cuda.synchronize()
            rb, vb = rb.cpu().numpy(), vb.cpu().numpy()
        else:
            rb, vb = np.empty((n, 3)), np.empty((n, 3))
            lbp.lbp_step_exchange(hb, f, rb if k != 4 else None, vb)
            if k == 4:
                lbp.lbp_particles_read(hb, r=rb)
        assert np.array_equal(ra, rb) and np.array_equal(va, vb), k
    assert lbp.lbp_get_step_index(hb) == 6
    fa, fb = gpu_pops(ha), gpu_pops(hb)
    assert np.array_equal(fa, fb)
    lbp.lbp_destroy(ha)
    lbp.lbp_destroy(hb)


def test_step_exchange_with_page_locked_buffers_equals_the_separate_calls():
    """With page-locked host buffers lbp_step_exchange replays copies + step as
    one graph per buffer parity; it stays bitwise equal to the separate calls
    across two alternating buffer sets, f_ext = None (previous forces kept), a
    parameter change between steps, and a VACF run whose 64-sample blocks are
    forked mid-way."""
    shape = (12, 13, 14)
    ps = wl.uniform_particles(7, shape, 8.0, 0.5, wl.stokes_radius(0.5, 0.8), 1e-4, 3, 5)
    ha = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=4)
    hb = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=4)
    K = 20
    for h in (ha, hb):
        lbp.lbp_vacf_configure(h, K)
    n = ps.n
    pin = lambda: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    sets = [(pin(), pin(), pin()), (pin(), pin(), pin())]
    g = np.random.default_rng(2)
    for k in range(150):
        keep = k % 7 == 6
        f = g.normal(0, 1e-5, (n, 3))
        fb, rb, vb = sets[(k // 3) % 2]
        if k == 90:  # an edit between steps drops the cached graphs
            for h in (ha, hb):
                lbp.lbp_particles_set_params(h, kT=2e-4, seed=4)
        if not keep:
            lbp.lbp_particles_set_external_force(ha, f)
        lbp.lbp_step(ha, 1)
        ra, va = np.empty((n, 3)), np.empty((n, 3))
        lbp.lbp_particles_read(ha, r=ra, v=va)
        fb[:] = f
        lbp.lbp_step_exchange(hb, None if keep else fb, rb, vb)
        assert np.array_equal(ra, rb) and np.array_equal(va, vb), k
    assert lbp.lbp_get_step_index(hb) == 150
    assert np.array_equal(gpu_pops(ha), gpu_pops(hb))
    ca, na = np.zeros(K + 1), np.zeros(K + 1, np.int64)
    cb, nb = np.zeros(K + 1), np.zeros(K + 1, np.int64)
    lbp.lbp_vacf_read(ha, ca, na)
    lbp.lbp_vacf_read(hb, cb, nb)
    assert na[0] > 0 and np.array_equal(na, nb) and np.array_equal(ca, cb)
    for h in (ha, hb):
        lbp.lbp_destroy(h)


def test_step_exchange_with_one_output_buffer():
    """Page-locked exchange asking for positions only, then velocities only: the
    particle kernel writes just the requested host buffer, and the run stays
    bitwise equal to the separate calls."""
    shape = (10, 9, 8)
    ps = wl.uniform_particles(5, shape, 8.0, 0.5, wl.stokes_radius(0.5, 0.8), 1e-4, 7, 8)
    ha = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=6)
    hb = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=6)
    n = ps.n
    rb = torch.full((n, 3), np.nan, dtype=torch.float64, pin_memory=True).numpy()
    vb = torch.full((n, 3), np.nan, dtype=torch.float64, pin_memory=True).numpy()
    for k in range(12):
        lbp.lbp_step(ha, 1)
        ra, va = np.empty((n, 3)), np.empty((n, 3))
        lbp.lbp_particles_read(ha, r=ra, v=va)
        if k < 6:
            lbp.lbp_step_exchange(hb, None, rb, None)
            assert np.array_equal(ra, rb), k
            assert np.all(np.isnan(vb)), k
        else:
            lbp.lbp_step_exchange(hb, None, None, vb)
            assert np.array_equal(va, vb), k
    assert np.array_equal(gpu_pops(ha), gpu_pops(hb))
    # the step index set back to the last exchanged step, whose index the
    # completion flag still holds: the call must still wait for the new step
    back = lbp.lbp_get_step_index(hb) - 1
    for h in (ha, hb):
        lbp.lbp_set_step_index(h, back)
    for k in range(3):
        lbp.lbp_step(ha, 1)
        ra = np.empty((n, 3))
        lbp.lbp_particles_read(ha, r=ra)
        lbp.lbp_step_exchange(hb, None, rb, None)
        assert np.array_equal(ra, rb), k
    for h in (ha, hb):
        lbp.lbp_destroy(h)


@pytest.mark.parametrize("device", [False, True])
def test_step_exchange_with_many_particles(device):
    """Enough particles for the thread-per-particle layout of the fit (48 or
    more per SM), with a partial last block and some pinned particles: the
    blocks write positions and velocities to the page-locked (or device)
    buffers as contiguous spans read back from the particle state, and the run
    stays bitwise equal to the separate calls, with both outputs and with one,
    with new external forces in some steps and the previous ones kept in
    others."""
    n = 48 * torch.cuda.get_device_properties(0).multi_processor_count + 35
    shape = (64, 64, 64)
    ps = wl.uniform_particles(n, shape, 8.0, 0.5, wl.stokes_radius(0.5, 0.8), 1e-4, 11, 12)
    pinned = np.zeros(n, np.uint8)
    pinned[::97] = 1
    pinned[-1] = 1
    ha = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=8)
    hb = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=8)
    f = np.random.default_rng(3).normal(0, 1e-5, (n, 3))
    for h in (ha, hb):
        lbp.lbp_particles_set_external_force(h, f, pinned)
    assert not lbp.lbp_diagnostics(hb)["fit_per_corner"]
    if device:
        buf = lambda: torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
        host = lambda x: (torch.cuda.synchronize(), x.cpu().numpy())[1]
        fb = buf()
    else:
        buf = lambda: torch.full((n, 3), np.nan, dtype=torch.float64, pin_memory=True).numpy()
        host = lambda x: x
        fb = buf()
    rb, vb = buf(), buf()
    g = np.random.default_rng(4)
    for k in range(8):
        fk = None if k % 3 == 2 else g.normal(0, 1e-5, (n, 3))
        if fk is not None:
            lbp.lbp_particles_set_external_force(ha, fk, pinned)  # NULL pinned would unpin
            fb[:] = torch.tensor(fk, device="cuda") if device else fk
        lbp.lbp_step(ha, 1)
        ra, va = np.empty((n, 3)), np.empty((n, 3))
        lbp.lbp_particles_read(ha, r=ra, v=va)
        if k < 6:
            lbp.lbp_step_exchange(hb, None if fk is None else fb, rb, vb)
            assert np.array_equal(va, host(vb)), k
        else:
            lbp.lbp_step_exchange(hb, None if fk is None else fb, rb, None)
        assert np.array_equal(ra, host(rb)), k
    assert np.array_equal(host(rb)[pinned == 1], ps.r[pinned == 1])
    assert np.array_equal(gpu_pops(ha), gpu_pops(hb))
    for h in (ha, hb):
        lbp.lbp_check(h)
        lbp.lbp_destroy(h)


def test_set_fluid_is_the_equilibrium_of_eq17():
    """lbp_set_fluid(rho, u) sets f = f^eq(rho~, u) at every node (oracle's Eq. 17)."""
    shape = (5, 6, 7)
    nz, ny, nx = shape
    N = nx * ny * nz
    g = np.random.default_rng(4)
    rho = 1.0 + 0.01 * g.uniform(-1, 1, N)
    u = 0.02 * g.uniform(-1, 1, (3, N))
    h = gpu_sim(shape, 0.8)
    lbp.lbp_set_fluid(h, rho, u)
    f = gpu_pops(h).reshape(15, N)
    want = np.stack([oracle.feq(rho[i], u[:, i]) for i in range(N)], axis=1)
    assert np.max(np.abs(f - want)) <= 1e-7 * np.max(np.abs(want - W[:, None]))
    lbp.lbp_set_fluid(h, None, None)
    assert np.array_equal(gpu_pops(h), np.broadcast_to(W4, (15,) + shape))
    lbp.lbp_destroy(h)


@pytest.mark.parametrize("graphs", [True, False])
def test_uniform_body_force_with_pinned_particle(graphs):
    """Eq. 18 with a uniform body force on every node plus a pinned particle's
    reaction force: a uniform flow driven past a held sphere, 80 steps."""
    shape = (12, 13, 15)
    ps = wl.uniform_particles(3, shape, 10.0, 0.5, wl.stokes_radius(0.5, 0.6), 0.0, 5, 6)
    G = np.array([2e-6, -1e-6, 5e-7])
    pinned = np.array([1, 0, 0], np.uint8)
    h = gpu_sim(shape, 0.6, ps, graphs=graphs)
    o = oracle_sim(shape, 0.6, ps)
    lbp.lbp_set_body_force(h, G)
    o.set_body_force(G)
    lbp.lbp_particles_set_external_force(h, None, pinned)
    o.set_external(None, pinned)
    lbp.lbp_step(h, 80)
    o.step(80)
    r, V, FH, FR = gpu_particles(h)
    ro, Vo, FHo, FRo = o.particles()
    assert np.array_equal(r[0], ps.r[0]) and np.array_equal(V[0], ps.V[0])
    assert np.max(np.abs(V - Vo)) <= 1e-5 * np.max(np.abs(Vo))
    assert np.max(np.abs(FH - FHo)) <= 1e-5 * np.max(np.abs(FHo))
    fo = o.fhat()
    assert np.max(np.abs(gpu_pops(h) - fo)) <= 1e-5 * dev_scale(fo) + F64_FLOOR
    # the body force did drive a flow: mean momentum close to 80 G less the drag
    rho, u, _ = o.fields()
    assert np.all(np.sign(u.reshape(3, -1).mean(1)) == np.sign(G))
    lbp.lbp_check(h)


@pytest.mark.parametrize("shape,n", [((3, 4, 5), 60), ((6, 5, 130), 400)])
def test_dense_particles_overflow_the_force_records(shape, n):
    """Many particles per 128-node row segment: shares beyond a segment's 8
    record slots take the overflow path; the result must still match the
    oracle and be bit-reproducible."""
    ps = wl.uniform_particles(n, shape, 10.0, 0.5, 0.2, 1e-4, 31, 32)
    outs = []
    for graphs in (True, False):
        h = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=4, graphs=graphs)
        lbp.lbp_step(h, 25)
        outs.append((gpu_pops(h), gpu_particles(h)))
        assert lbp.lbp_diagnostics(h)["overflow_shares"] > 0  # the overflow path ran
        lbp.lbp_check(h)
        lbp.lbp_destroy(h)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1][1], outs[1][1][1])
    o = oracle_sim(shape, 0.8, ps, kT=1e-4, seed=4)
    o.step(25)
    fo = o.fhat()
    _, Vo, _, _ = o.particles()
    assert np.max(np.abs(outs[0][0] - fo)) <= 1e-5 * dev_scale(fo) + F64_FLOOR
    assert np.max(np.abs(outs[0][1][1] - Vo)) <= 1e-5 * np.max(np.abs(Vo))


def test_pinned_particle_and_external_force():
    shape = (10, 10, 10)
    r = np.array([[5.5, 5.5, 5.5], [2.3, 7.1, 4.4]])
    ps = wl.ParticleSet(r, np.array([[0.0, 0, 0], [0.001, 0, 0.002]]), np.array([10.0, 5.0]),
                        np.array([0.5, 0.3]), np.array([0.26, 0.2]))
    f0 = np.broadcast_to(np.stack([oracle.feq(1.0, np.array([1e-3, 0, 0]))], 1)[:, :, None, None],
                         (15,) + shape).copy()
    fext = np.array([[0.0, 0, 0], [1e-5, -2e-5, 0]])
    pin = np.array([1, 0], np.uint8)
    h = gpu_sim(shape, 0.8, ps)
    lbp.lbp_set_populations(h, f0)
    lbp.lbp_particles_set_external_force(h, fext, pin)
    o = oracle_sim(shape, 0.8, ps)
    o.set_fhat(f0)
    o.set_external(fext, pin)
    lbp.lbp_step(h, 40)
    o.step(40)
    rg, Vg, FHg, _ = gpu_particles(h)
    ro, Vo, FHo, _ = o.particles()
    assert np.array_equal(rg[0], r[0]) and np.array_equal(Vg[0], [0, 0, 0])
    # FP32 rounding of the 1e-3 background flow sets the error scale: compare
    # each particle's force and velocity against its own magnitude
    for i in range(2):
        assert np.max(np.abs(FHg[i] - FHo[i])) <= 1e-5 * np.max(np.abs(FHo[i]))
        assert np.max(np.abs(Vg[i] - Vo[i])) <= 1e-5 * max(np.max(np.abs(Vo[i])), 1e-30)


def test_momentum_budget_on_gpu():
    shape = (12, 12, 12)
    ps = wl.uniform_particles(20, shape, 8.0, 0.4, 0.2, 1e-4, 5, 6)
    h = gpu_sim(shape, 0.75, ps, kT=1e-4, seed=3)

    def P():
        f = gpu_pops(h)
        _, V, _, _ = gpu_particles(h)
        return E.T.astype(float) @ f.reshape(15, -1).sum(1) + (ps.M[:, None] * V).sum(0)

    P0 = P()
    inj = np.zeros(3)
    for _ in range(20):
        lbp.lbp_step(h, 1)
        inj += gpu_particles(h)[3].sum(0)
    # fluid momentum carries FP32 rounding of ~1e-8 per node population
    assert np.allclose(P() - P0, inj, atol=1e-9)


def test_deterministic_and_graph_invariant():
    shape = (10, 12, 14)
    ps = wl.uniform_particles(60, shape, 10.0, 0.5, 0.26, 1e-4, 8, 9)
    outs = []
    for graphs in (True, False, True):
        h = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=5, graphs=graphs)
        lbp.lbp_step(h, 30)
        outs.append((gpu_pops(h), gpu_particles(h)[1]))
        lbp.lbp_destroy(h)
    for f, V in outs[1:]:
        assert np.array_equal(f, outs[0][0])
        assert np.array_equal(V, outs[0][1])


# ---------------------------------------------------------------- VACF
def test_vacf_matches_oracle_on_the_same_trajectory():
    shape = (8, 8, 8)
    ps = wl.uniform_particles(37, shape, 6.0, 0.5, 0.2, 1e-4, 1, 2)
    h = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=2)
    K = 90
    lbp.lbp_vacf_configure(h, K)
    traj = []
    T = 150  # two full 64-sample blocks and a partial one
    for _ in range(T):
        lbp.lbp_step(h, 1)
        traj.append(gpu_particles(h)[1])
    cs = np.empty(K + 1)
    cnt = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, cs, cnt)
    ref, refc = oracle.vacf(np.array(traj, np.float32).astype(np.float64), K)
    assert np.array_equal(cnt, refc)
    assert np.max(np.abs(cs - ref)) <= 1e-6 * ref[0]
    check_msd(h, traj, K)
    # reading again after more steps continues the same sums (the flush above
    # left the next blocks starting at sample 150, not at a multiple of 64)
    for _ in range(70):
        lbp.lbp_step(h, 1)
        traj.append(gpu_particles(h)[1])
    lbp.lbp_vacf_read(h, cs, cnt)
    ref, refc = oracle.vacf(np.array(traj, np.float32).astype(np.float64), K)
    assert np.array_equal(cnt, refc)
    assert np.max(np.abs(cs - ref)) <= 1e-6 * ref[0]
    check_msd(h, traj, K)


# FP32 products summed over components by the tensor cores, then FP64: the MSD
# of the GPU's own (FP32) velocity samples within this relative error
MSD_REL = 2e-6


def check_msd(h, traj, K, rel=MSD_REL):
    """The library's mean squared displacement against the oracle's, evaluated on
    positions X(t) = sum_{s <= t} V(s) of the same FP32 velocity samples (the
    displacement X(t0 + k) - X(t0) is the sum of the k velocities after t0, Eq. 2)."""
    ms = np.empty(K + 1)
    mc = np.empty(K + 1, np.int64)
    lbp.lbp_msd_read(h, ms, mc)
    V = np.array(traj, np.float32).astype(np.float64)
    ref, refc = oracle.msd(np.cumsum(V, axis=0), K)
    assert np.array_equal(mc, refc)
    assert ms[0] == 0.0
    T = min(len(traj), K + 1)  # lags with at least one origin
    assert np.all(ms[T:] == 0.0)
    err = np.abs(ms[1:T] - ref[1:T]) / ref[1:T]
    assert np.max(err) <= rel, (np.max(err), int(np.argmax(err)) + 1)


def test_vacf_spans_lag_tiles_and_component_chunks_with_ragged_tails():
    """The block correlation with several 128-lag tiles and 1024-component
    chunks, both ragged (K = 300: 128 + 128 + 45 lags; 400 particles: 1024 +
    176 components), three full 64-sample blocks and a partial one flushed by
    the read: sums within 1e-6 of C(0) of the oracle's FP64 correlation of the
    same (FP32) trajectory, pair counts exact."""
    shape = (16, 20, 24)
    ps = wl.uniform_particles(400, shape, 6.0, 0.5, 0.2, 1e-4, 5, 6)
    h = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=3)
    K = 300
    lbp.lbp_vacf_configure(h, K)
    traj = []
    for _ in range(3 * 64 + 37):
        lbp.lbp_step(h, 1)
        traj.append(gpu_particles(h)[1])
    cs = np.empty(K + 1)
    cnt = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, cs, cnt)
    ref, refc = oracle.vacf(np.array(traj, np.float32).astype(np.float64), K)
    assert np.array_equal(cnt, refc)
    assert np.max(np.abs(cs - ref)) <= 1e-6 * ref[0]
    check_msd(h, traj, K)
    lbp.lbp_destroy(h)


def test_msd_is_not_kept_per_particle():
    shape = (8, 8, 8)
    ps = wl.uniform_particles(5, shape, 6.0, 0.5, 0.2, 1e-4, 1, 2)
    h = gpu_sim(shape, 0.8, ps, kT=1e-4, seed=2)
    lbp.lbp_vacf_configure_ex(h, 20, 1)
    lbp.lbp_step(h, 5)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_msd_read(h, np.empty(21), np.empty(21, np.int64))
    assert ei.value.status == lbp.LBP_ESTATE


def test_vacf_configure_refuses_oversized_buffers_without_allocating():
    """A VACF whose buffers would pass 64 GiB (lbp_vacf_configure), or a
    per-particle VACF past its limits, is refused before anything is
    allocated: LBP_EINVAL, the VACF off, device memory unchanged, and the
    handle steps on.  A large accepted configuration then correlates the few
    samples taken (pair counts exact, lags beyond the samples zero)."""
    shape = (16, 16, 16)
    h = lbp.lbp_create(16, 16, 16, 0.8)
    ps = wl.uniform_particles(3000, shape, 6.0, 0.5, 0.2, 1e-4, 1, 2)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=1e-4, seed=3)
    lbp.lbp_vacf_configure(h, 16)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # ~36 KB of ring and ~6 KB of sums and correlation buffers per lag
    for call in (lambda: lbp.lbp_vacf_configure(h, 2_000_000),
                 lambda: lbp.lbp_vacf_configure_ex(h, 100_000, True)):
        with pytest.raises(lbp.LbpError) as ei:
            call()
        assert ei.value.status == lbp.LBP_EINVAL
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_vacf_read(h, np.empty(17), np.empty(17, np.int64))
    assert ei.value.status == lbp.LBP_ESTATE
    lbp.lbp_step(h, 2)
    lbp.lbp_check(h)
    K = 200_000  # ~8.4 GB of buffers
    lbp.lbp_vacf_configure(h, K)
    lbp.lbp_step(h, 3)
    cs, ct = np.empty(K + 1), np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, cs, ct)
    lbp.lbp_check(h)
    assert list(ct[:4]) == [9000, 6000, 3000, 0] and not np.any(ct[4:]) and not np.any(cs[3:])
    assert cs[0] > 0
    lbp.lbp_destroy(h)


def test_kernel_timing_counts_launches_and_changes_no_result():
    """lbp_timing_enable / lbp_timing_read: one timed stream-collide launch per
    step (plain launches with events instead of the graph), a positive total
    duration, the counter restarted by a new enable; the populations and
    particles equal, bit for bit, those of the same run with timing off."""
    shape = (12, 10, 24)

    def make():
        h = lbp.lbp_create(24, 10, 12, 0.7)
        lbp.lbp_set_populations(h, wl.perturbed_populations(W, shape, 0.02, 4))
        ps = wl.uniform_particles(7, shape, 6.0, 0.5, 0.2, 1e-4, 5, 6)
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=1e-4, seed=2)
        return h
    ha, hb = make(), make()
    lbp.lbp_timing_enable(ha, True)
    lbp.lbp_step(ha, 11)
    ms, n = lbp.lbp_timing_read(ha)
    assert n == 11 and 0.0 < ms < 1e4
    lbp.lbp_timing_enable(ha, True)
    lbp.lbp_step(ha, 4)
    assert lbp.lbp_timing_read(ha)[1] == 4
    lbp.lbp_timing_enable(ha, False)
    lbp.lbp_step(ha, 5)
    lbp.lbp_step(hb, 20)
    outs = []
    for h in (ha, hb):
        lbp.lbp_check(h)
        f = np.empty((15,) + shape)
        lbp.lbp_read_populations(h, f)
        r, v = np.empty((7, 3)), np.empty((7, 3))
        lbp.lbp_particles_read(h, r, v)
        outs.append((f, r, v))
        lbp.lbp_destroy(h)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_vacf_requires_particles():
    h = gpu_sim((4, 4, 4), 0.8)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_vacf_configure(h, 10)
    assert ei.value.status == lbp.LBP_ESTATE


# ---------------------------------------------------------------- validation on device
def test_particle_validation():
    h = gpu_sim((8, 8, 8), 0.8)
    bad = [
        (np.array([[8.0, 1, 1]]), np.zeros((1, 3)), [1.0], [0.5], [0.2]),   # outside the box
        (np.array([[1.0, 1, 1]]), np.full((1, 3), np.nan), [1.0], [0.5], [0.2]),
        (np.array([[1.0, 1, 1]]), np.zeros((1, 3)), [0.0], [0.5], [0.2]),   # mass
        (np.array([[1.0, 1, 1]]), np.zeros((1, 3)), [1.0], [0.5], [2.0]),   # R > sqrt(3)
    ]
    for r, v, m, g, R in bad:
        with pytest.raises(lbp.LbpError) as ei:
            lbp.lbp_particles_add(h, r, v, np.array(m), np.array(g), np.array(R))
        assert ei.value.status == lbp.LBP_EINVAL
    assert h.np == 0
    lbp.lbp_particles_add(h, np.array([[1.0, 1, 1]]), np.zeros((1, 3)), np.array([1.0]),
                          np.array([0.5]), np.array([1.0]))
    with pytest.raises(lbp.LbpError):
        lbp.lbp_particles_set_params(h, fit_exclude_inside=1)  # R = 1 > sqrt(3)/2
    with pytest.raises(lbp.LbpError):
        lbp.lbp_particles_set_params(h, kT=-1.0)


def test_volume_fraction_and_the_dense_suspension_warning():
    """Section 2.2: the method was checked below a volume fraction of 0.1.
    lbp_volume_fraction gives sum(4/3 pi R^3) / nodes per box (-1: the largest),
    R from Stokes' law where no radius is given; a denser suspension is
    accepted, with a warning from the binding."""
    sphere = 4.0 / 3.0 * math.pi
    h = lbp.lbp_create_batch([(16, 16, 16, 0.8), (8, 8, 8, 0.8)])
    g = np.random.default_rng(5)
    with warnings.catch_warnings(record=True) as seen:
        warnings.simplefilter("always")
        lbp.lbp_particles_add_to(h, 0, g.random((10, 3)) * 16, np.zeros((10, 3)), np.full(10, 10.0),
                                 np.full(10, 0.5), np.full(10, 1.0))
    assert not [w for w in seen if "volume fraction" in str(w.message)]  # below 0.1: none
    assert lbp.lbp_volume_fraction(h, 0) == pytest.approx(10 * sphere / 4096, rel=1e-12)
    assert lbp.lbp_volume_fraction(h, 1) == 0.0
    with pytest.warns(RuntimeWarning, match="volume fraction"):
        lbp.lbp_particles_add_to(h, 1, g.random((13, 3)) * 8, np.zeros((13, 3)), np.full(13, 10.0),
                                 np.full(13, 0.5), np.full(13, 1.0))
    assert h.np == 23
    assert lbp.lbp_volume_fraction(h, 1) == pytest.approx(13 * sphere / 512, rel=1e-12)
    assert lbp.lbp_volume_fraction(h, -1) == pytest.approx(13 * sphere / 512, rel=1e-12)
    for bad in (2, -2):
        with pytest.raises(lbp.LbpError) as ei:
            lbp.lbp_volume_fraction(h, bad)
        assert ei.value.status == lbp.LBP_EINVAL
    lbp.lbp_destroy(h)
    h = gpu_sim((16, 16, 16), 0.8)
    lbp.lbp_particles_add(h, g.random((5, 3)) * 16, np.zeros((5, 3)), np.full(5, 10.0), np.full(5, 0.5))
    R = 0.5 / (6 * math.pi * 0.1)
    assert lbp.lbp_volume_fraction(h) == pytest.approx(5 * sphere * R ** 3 / 4096, rel=1e-12)
    lbp.lbp_destroy(h)


def test_stokes_radius_default():
    h = gpu_sim((8, 8, 8), 0.8)
    r = np.array([[4.5, 4.5, 4.5]])
    lbp.lbp_particles_add(h, r, np.array([[0.01, 0, 0]]), np.array([10.0]), np.array([0.5]))
    lbp.lbp_step(h, 1)
    _, _, FH, _ = gpu_particles(h)
    R = 0.5 / (6 * math.pi * 0.1)
    U, _ = oracle.stokeslet_fit(oracle.corners(r[0])[1], np.zeros((8, 3)), np.array([0.01, 0, 0]), R)
    assert FH[0, 0] == pytest.approx(-0.5 * U, rel=1e-6)


def test_nan_watchdog():
    h = gpu_sim((8, 8, 8), 0.8)
    lbp.lbp_particles_add(h, np.array([[4.5, 4.5, 4.5]]), np.zeros((1, 3)), np.array([1.0]),
                          np.array([0.5]), np.array([0.2]))
    lbp.lbp_particles_set_external_force(h, np.array([[np.inf, 0.0, 0.0]]))
    lbp.lbp_step(h, 1)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_check(h)
    assert ei.value.status == lbp.LBP_ENAN
    r = np.empty((1, 3))
    lbp.lbp_particles_read(h, r=r)
    assert np.all((r >= 0) & (r < 8))
    lbp.lbp_check(h)  # the flag is cleared once reported


# ---------------------------------------------------------------- reduced-precision storage
@pytest.mark.parametrize("prec,tol", [(lbp.LBP_BF16, 8e-3), (lbp.LBP_F16, 1e-3)])
def test_reduced_precision_one_step(prec, tol):
    """BF16 keeps 8 mantissa bits (rounding <= 2^-9 of g per store), scaled FP16 keeps
    11 (<= 2^-11): the input rounding plus the output rounding bound one step."""
    shape = (13, 21, 300)
    f0 = wl.perturbed_populations(W, shape, 0.05, 17)
    h = lbp.lbp_create(300, 21, 13, 0.8, precision=prec)
    lbp.lbp_set_populations(h, f0)
    lbp.lbp_step(h, 1)
    o = oracle_sim(shape, 0.8)
    o.set_fhat(f0)
    o.step(1)
    fo = o.fhat()
    assert np.max(np.abs(gpu_pops(h) - fo)) <= tol * dev_scale(fo)


@pytest.mark.parametrize("prec,tol_v,tol_u", [(lbp.LBP_F32, 1e-5, 1e-5), (lbp.LBP_F16, 1e-4, 1e-3),
                                              (lbp.LBP_BF16, 1e-3, 5e-3)])
def test_reduced_precision_subrun_error(prec, tol_v, tol_u):
    """The 64^3 subrun of the 256^3 storage comparison (256 particles, same number
    density, kT = 1e-4), 300 steps against the FP64 oracle.  Measured on GB300 after
    1000 steps (max relative error): particle V 5.7e-6 (F32), 3.8e-5 (F16), 1.9e-4
    (BF16); fluid u 7.3e-6, 2.9e-4, 1.8e-3."""
    w = wl.BROWNIAN_64
    ps = w.particles()
    nz, ny, nx = w.shape_zyx
    h = lbp.lbp_create(nx, ny, nz, w.tau, precision=prec)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=w.kT, seed=3)
    lbp.lbp_step(h, 300)
    o = oracle_sim(w.shape_zyx, w.tau, ps, kT=w.kT, seed=3)
    o.step(300)
    _, Vo, _, _ = o.particles()
    _, uo, _ = o.fields()
    V = np.empty((ps.n, 3))
    lbp.lbp_particles_read(h, v=V)
    u = np.empty(3 * w.nodes)
    lbp.lbp_read_fields(h, u=u)
    assert np.max(np.abs(V - Vo)) <= tol_v * np.max(np.abs(Vo))
    assert np.max(np.abs(u.reshape(uo.shape) - uo)) <= tol_u * np.max(np.abs(uo))
    lbp.lbp_check(h)


# ---------------------------------------------------------------- full size
@pytest.mark.parametrize("prec,tol_v,tol_f", [(lbp.LBP_F32, 1e-5, 1e-5), (lbp.LBP_BF16, 2e-2, 1e-2),
                                              (lbp.LBP_F16, 2e-3, 2e-3)])
def test_full_size_bench_workload_against_the_oracle(prec, tol_v, tol_f):
    """The bench workload at its full size (256^3, 16384 Brownian particles,
    kT = 1e-4) in the launch configuration the bench times (autotuned kernel
    shape, CUDA graphs, VACF accumulating to lag 5000), two steps from a
    perturbed state, against the FP64 oracle: every particle's F_R bit for bit,
    F_H, V and r within the stated tolerance, and populations on 200000
    sampled nodes.  Tolerances per storage type: FP32 as the small-box tests;
    BF16 and FP16 at their measured one-step storage errors (BF16 3.9e-3,
    FP16 4.8e-4 of the deviation scale on the 64^3 subrun)."""
    w = wl.BROWNIAN_256
    nz, ny, nx = w.shape_zyx
    ps = w.particles()
    f0 = wl.perturbed_populations(W, w.shape_zyx, 0.01, 31)
    h = lbp.lbp_create(nx, ny, nz, w.tau, precision=prec)
    lbp.lbp_set_populations(h, f0)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=w.kT, seed=w.seed_noise)
    lbp.lbp_vacf_configure(h, 5000)
    lbp.lbp_autotune(h, 3)
    # the oracle starts from what the GPU stores (the 2-byte types round f0)
    fs = gpu_pops(h)
    o = oracle_sim(w.shape_zyx, w.tau, ps, kT=w.kT, seed=w.seed_noise)
    o.set_fhat(fs)
    del fs
    lbp.lbp_step(h, 2)
    o.step(2)
    r, V, FH, FR = gpu_particles(h)
    ro, Vo, FHo, FRo = o.particles()
    assert np.array_equal(FR, FRo)
    assert np.max(np.abs(V - Vo)) <= tol_v * np.max(np.abs(Vo))
    assert np.max(np.abs(FH - FHo)) <= tol_v * np.max(np.abs(FHo))
    d = np.abs(r - ro)
    d = np.minimum(d, np.array([nx, ny, nz], float) - d)
    assert np.max(d) <= tol_v
    f = gpu_pops(h).reshape(15, -1)
    fo = o.fhat().reshape(15, -1)
    o.close()
    idx = np.random.default_rng(5).choice(f.shape[1], 200000, replace=False)
    scale = np.max(np.abs(fo[:, idx] - W[:, None]))
    assert np.max(np.abs(f[:, idx] - fo[:, idx])) <= tol_f * scale + F64_FLOOR
    lbp.lbp_check(h)
    lbp.lbp_destroy(h)


def test_full_size_vacf_run_against_its_own_trajectory():
    """The VACF run at its full size (128^3, 2000 Brownian particles, lag 5000),
    6000 steps: the library's VACF sums equal the all-origins correlation of the
    trajectory read back step by step (FP32 velocities, products summed in FP64
    by FFT), to 1e-5 of C(0); pair counts exact."""
    w = wl.BROWNIAN_128
    nz, ny, nx = w.shape_zyx
    ps = w.particles()
    K, T = w.vacf_lag, 6000
    h = lbp.lbp_create(nx, ny, nz, w.tau)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=w.kT, seed=w.seed_noise)
    lbp.lbp_vacf_configure(h, K)
    lbp.lbp_autotune(h, 3)
    n = ps.n
    traj = np.empty((T, n, 3), np.float32)
    V = np.empty((n, 3))
    for t in range(T):
        lbp.lbp_step_exchange(h, None, None, V)
        traj[t] = V
    cs = np.empty(K + 1)
    cnt = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, cs, cnt)
    ms = np.empty(K + 1)
    mc = np.empty(K + 1, np.int64)
    lbp.lbp_msd_read(h, ms, mc)
    lbp.lbp_check(h)
    lbp.lbp_destroy(h)
    x = traj.reshape(T, 3 * n).astype(np.float64)
    L = 1 << int(np.ceil(np.log2(2 * T)))
    F = np.fft.rfft(x, n=L, axis=0)
    ref = np.fft.irfft((F * np.conj(F)).sum(axis=1), n=L)[:K + 1]
    assert np.array_equal(cnt, n * (T - np.arange(K + 1)))
    assert np.max(np.abs(cs - ref)) <= 1e-5 * ref[0]
    # MSD of the positions X(t) = sum_{s <= t} V(s): sum_t0 |X(t0+k)|^2 + |X(t0)|^2
    # - 2 X(t0+k).X(t0), the cross term by FFT (FP64)
    X = np.cumsum(x, axis=0)
    X -= X[T // 2]  # centre the positions to keep the FFT's cancellation small
    s2 = (X * X).sum(axis=1)
    c2 = np.concatenate([[0.0], np.cumsum(s2)])
    FX = np.fft.rfft(X, n=L, axis=0)
    cross = np.fft.irfft((FX * np.conj(FX)).sum(axis=1), n=L)[:K + 1]
    k = np.arange(K + 1)
    mref = (c2[T] - c2[k]) + c2[T - k] - 2.0 * cross
    assert np.array_equal(mc, cnt)
    rel = np.abs(ms[1:] - mref[1:]) / mref[1:]
    assert np.max(rel) <= 1e-4, (np.max(rel), int(np.argmax(rel)) + 1)


def test_full_size_ensemble_equals_its_boxes_alone():
    """The ensemble at its full size (48 x 64^3 + 16 x 96^3 + 4 x 160^3, one
    Brownian particle each, tau in {0.6, 0.8, 1.0}), in the bench's launch
    configuration (autotuned shape, graphs, per-particle VACF), five steps:
    every box and its particle bitwise equal to the same box run alone (box 0,
    whose particle has index 0 in both, with the random force on; the others
    with kT = 0, since a particle's Philox counter is its index in the handle)."""
    e = wl.ENSEMBLE_68
    steps = 5
    for kT in (e.kT, 0.0):
        h = lbp.lbp_create_batch(e.boxes)
        for b in range(len(e.boxes)):
            p = e.particles(b)
            lbp.lbp_particles_add_to(h, b, p.r, p.V, p.M, p.gamma, p.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=e.seed_noise)
        lbp.lbp_vacf_configure_ex(h, 5000, 1)
        lbp.lbp_autotune(h, 3)
        lbp.lbp_step(h, steps)
        f = np.empty((15, h.N))
        lbp.lbp_read_populations(h, f)
        V = np.empty((len(e.boxes), 3))
        lbp.lbp_particles_read(h, v=V)
        lbp.lbp_destroy(h)
        off = 0
        for b, (bx, by, bz, tau) in enumerate(e.boxes):
            nb = bx * by * bz
            if (kT > 0) == (b == 0):
                p = e.particles(b)
                hs = lbp.lbp_create(bx, by, bz, tau)
                lbp.lbp_particles_add(hs, p.r, p.V, p.M, p.gamma, p.R)
                lbp.lbp_particles_set_params(hs, kT=kT, seed=e.seed_noise)
                lbp.lbp_step(hs, steps)
                fs = np.empty((15, nb))
                lbp.lbp_read_populations(hs, fs)
                Vs = np.empty((1, 3))
                lbp.lbp_particles_read(hs, v=Vs)
                lbp.lbp_destroy(hs)
                assert np.array_equal(f[:, off:off + nb], fs), b
                assert np.array_equal(V[b], Vs[0]), b
            off += nb
