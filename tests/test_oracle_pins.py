"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks retypes an oracle formula: each compares the oracle with
a textbook identity, a closed form, an independent library routine (numpy's
Philox, numpy least squares, numpy correlation), a conservation law or a
special case solved by hand.  Citations are to arXiv:1909.13412.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1909_13412_gb300 import workloads as wl

E, W = oracle.d3q15()
E = E.astype(np.float64)


# ------------------------------------------------------------ D3Q15 table (Section 2.2)
def test_d3q15_isotropy():
    """The lattice moments that recover Navier-Stokes (Succi's D3Q15 table)."""
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose((W[:, None] * E).sum(0), 0.0, atol=1e-16)
    second = np.einsum("a,ai,aj->ij", W, E, E)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", W, E, E, E), 0.0, atol=1e-16)
    assert (W * E[:, 0] ** 4).sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert (W * E[:, 0] ** 2 * E[:, 1] ** 2).sum() == pytest.approx(1.0 / 9.0, abs=1e-15)
    speeds = (E ** 2).sum(1)
    assert sorted(speeds.tolist()) == [0] + [1] * 6 + [3] * 8
    # every direction has its opposite
    for a in range(15):
        assert any(np.array_equal(E[b], -E[a]) for b in range(15))


# ------------------------------------------------------------ equilibrium (Eq. 17)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    """sum f^eq = rho~, sum e f^eq = u, sum e_i e_j f^eq = rho~ d_ij/3 + u_i u_j."""
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * g.standard_normal()
    u = 0.05 * g.standard_normal(3)
    fe = oracle.feq(rho, u)
    assert fe.sum() == pytest.approx(rho, abs=1e-15)
    assert np.allclose(E.T @ fe, u, atol=1e-16)
    P = np.einsum("ai,aj,a->ij", E, E, fe)
    assert np.allclose(P, rho * np.eye(3) / 3.0 + np.outer(u, u), atol=1e-15)


def test_equilibrium_at_rest_is_weights():
    assert np.allclose(oracle.feq(1.0, np.zeros(3)), W, atol=0)


# ------------------------------------------------------------ collision + force (Eqs. 14-19)
def test_collision_conserves_mass_and_adds_force():
    """BGK conserves rho~ and u; the force term adds exactly F to sum e f (Eq. 18-19)."""
    g = np.random.default_rng(5)
    shp = (2, 3, 4)
    f = wl.perturbed_populations(W, shp, 0.2, 7)
    rho, u = oracle.moments(f)
    F = 1e-3 * g.standard_normal((3,) + shp)
    fh = oracle.collide(f, rho, u, 0.7, F)
    rho2, u2 = oracle.moments(fh)
    assert np.allclose(rho2, rho, atol=1e-15)
    assert np.allclose(u2, u + F, atol=1e-15)
    fh0 = oracle.collide(f, rho, u, 0.7, None)
    # with f = f^eq the collision is the identity
    feq = np.stack([oracle.feq(rho[i, j, k], u[:, i, j, k]) for i in range(2) for j in range(3)
                    for k in range(4)], axis=1).reshape((15,) + shp)
    assert np.allclose(oracle.collide(feq, rho, u, 0.7, None), feq, atol=1e-16)
    # relaxation: f - fhat = (f - f^eq)/tau
    assert np.allclose(f - fh0, (f - feq) / 0.7, atol=1e-15)


def test_force_term_moments():
    """sum_a 3 w_a F.e_a = 0 and sum_a 3 w_a (F.e_a) e_a = F."""
    F = np.array([0.3, -0.2, 0.7])
    G = 3.0 * W * (E @ F)
    assert abs(G.sum()) < 1e-16
    assert np.allclose(E.T @ G, F, atol=1e-16)


# ------------------------------------------------------------ streaming (Eq. 20)
def test_streaming_moves_each_population_along_its_velocity():
    nz, ny, nx = 5, 6, 7
    for a in range(15):
        fh = np.zeros((15, nz, ny, nx))
        x0 = (2, 3, 4)  # (z, y, x)
        fh[a, x0[0], x0[1], x0[2]] = 1.0
        f = oracle.stream(fh)
        z1 = (x0[0] + int(E[a, 2])) % nz
        y1 = (x0[1] + int(E[a, 1])) % ny
        x1 = (x0[2] + int(E[a, 0])) % nx
        assert f[a, z1, y1, x1] == 1.0
        assert f.sum() == 1.0


def test_streaming_is_a_permutation():
    L = 6
    f0 = wl.perturbed_populations(W, (L, L, L), 0.5, 3)
    f = f0.copy()
    for _ in range(L):
        f = oracle.stream(f)
    assert np.array_equal(f, f0)


# ------------------------------------------------------------ whole fluid step
def test_uniform_states_are_fixed_points():
    for u in ([0, 0, 0], [0.02, -0.01, 0.005]):
        s = oracle.Sim(4, 5, 6, 0.8)
        fe = oracle.feq(1.01, np.array(u, float))
        s.set_fhat(np.broadcast_to(fe[:, None, None, None], (15, 6, 5, 4)).copy())
        s.step(5)
        assert np.allclose(s.fhat(), fe[:, None, None, None], atol=1e-16)


def test_mass_conservation_random_state():
    s = oracle.Sim(8, 6, 5, 0.62)
    f0 = wl.perturbed_populations(W, (5, 6, 8), 0.3, 11)
    s.set_fhat(f0)
    m0 = f0.sum()
    s.step(50)
    assert s.fhat().sum() == pytest.approx(m0, rel=1e-13)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_shear_wave_decays_at_lattice_viscosity(tau):
    """u_y = U sin(kx) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3 (Eq. 16)."""
    L = 64
    k = 2 * np.pi / L
    x = np.arange(L)
    f = np.stack([oracle.feq(1.0, np.array([0.0, 1e-4 * np.sin(k * xi), 0.0])) for xi in x],
                 axis=1).reshape(15, 1, 1, L)
    s = oracle.Sim(L, 1, 1, tau)
    s.set_fhat(f)
    amps = []
    for dt in (50, 200):
        s.step(dt)
        _, u, _ = s.fields()
        amps.append(2.0 / L * np.sum(u[1, 0, 0, :] * np.sin(k * x)))
    rate = np.log(amps[0] / amps[1]) / 200.0
    nu = (tau - 0.5) / 3.0
    assert rate == pytest.approx(nu * k * k, rel=2e-3)


# ------------------------------------------------------------ particle geometry (Eq. 9)
def test_corner_weights_reproduce_linear_functions():
    g = np.random.default_rng(4)
    for _ in range(20):
        r = g.uniform(0, 20, 3)
        base, d, Wp = oracle.corners(r)
        assert np.array_equal(base, np.floor(r).astype(np.int32))
        xp = d + r
        assert np.allclose(xp - np.round(xp), 0, atol=1e-13)
        assert np.all(np.abs(d) <= 1.0)
        assert Wp.sum() == pytest.approx(1.0, abs=1e-15)
        assert np.all(Wp >= 0)
        # trilinear interpolation of a linear field is exact -> sum W_p d_p = 0
        assert np.allclose((Wp[:, None] * d).sum(0), 0.0, atol=1e-14)


# ------------------------------------------------------------ Stokeslet fit (Eq. 8)
def _oseen_basis(d, e, R):
    """Uniform stream minus the Stokeslet of force 6 pi eta R e, written with the
    Oseen tensor (I/r + d d^T / r^3) -- an independent form of Eq. 8."""
    out = []
    for dp in d:
        r = np.linalg.norm(dp)
        G = np.eye(3) / r + np.outer(dp, dp) / r ** 3
        out.append(e - 0.75 * R * G @ e)
    return np.array(out)


@pytest.mark.parametrize("seed", range(6))
def test_stokeslet_fit_matches_least_squares(seed):
    g = np.random.default_rng(seed)
    r = g.uniform(3, 4, 3)
    _, d, _ = oracle.corners(r)
    uN = 1e-3 * g.standard_normal((8, 3))
    V = 1e-3 * g.standard_normal(3)
    R = g.uniform(0.1, 0.8)
    U, eN = oracle.stokeslet_fit(d, uN, V, R)
    w = uN - V
    e_ref = w.mean(0) / np.linalg.norm(w.mean(0))
    assert np.allclose(eN, e_ref, atol=1e-15)
    A = _oseen_basis(d, e_ref, R)
    sol, *_ = np.linalg.lstsq(A.reshape(-1, 1), w.reshape(-1), rcond=None)
    assert U == pytest.approx(sol[0], rel=1e-12, abs=1e-18)
    # and it is the minimiser: any other amplitude has a larger residual
    res = lambda x: np.sum((w - x * A) ** 2)
    assert res(U) <= min(res(U * (1 + 1e-6)), res(U * (1 - 1e-6)))


def test_stokeslet_fit_recovers_exact_stokes_flow():
    """With the particle at the cell centre and w_p = U0 u^A(d_p), the fit returns U0."""
    r = np.array([5.5, 5.5, 5.5])
    _, d, _ = oracle.corners(r)
    e = np.array([0.6, -0.48, 0.64])
    R, U0 = 0.3, 2.5e-3
    w = U0 * _oseen_basis(d, e, R)
    U, eN = oracle.stokeslet_fit(d, w, np.zeros(3), R)
    assert U == pytest.approx(U0, rel=1e-13)
    assert np.allclose(eN, e, atol=1e-14)


def test_stokeslet_fit_first_step_of_kicked_particle():
    """Fluid at rest, particle at a cell centre moving at V: every corner sees w = -V,
    r_p = sqrt(3)/2, (e.d_p)^2 = 1/4, and Eq. 8 reduces by hand to
    U/|V| = (c1 - 3R/(16 r^3)) / (c1^2 - 3R c1/(8 r^3) + 9R^2/(64 r^4)),
    c1 = 1 - 3R/(4r); at gamma = 0.5, tau = 0.8 (R = 0.26526) that is 1.40724."""
    R = wl.stokes_radius(0.5, 0.8)
    r = math.sqrt(3) / 2
    c1 = 1 - 3 * R / (4 * r)
    expect = (c1 - 3 * R / (16 * r ** 3)) / (c1 ** 2 - 3 * R * c1 / (8 * r ** 3) + 9 * R ** 2 / (64 * r ** 4))
    assert expect == pytest.approx(1.40724, abs=5e-6)
    _, d, _ = oracle.corners(np.array([16.5, 16.5, 16.5]))
    V = np.array([0.01, 0.0, 0.0])
    U, eN = oracle.stokeslet_fit(d, np.zeros((8, 3)), V, R)
    assert np.allclose(eN, [-1, 0, 0])
    assert U / 0.01 == pytest.approx(expect, rel=1e-13)
    # through the whole step: F_H = gamma U e^N
    s = oracle.Sim(32, 32, 32, 0.8)
    s.add_particles([[16.5, 16.5, 16.5]], [V], [10.0], [0.5], [R])
    s.set_params()
    s.step(1)
    _, V1, FH, FR = s.particles()
    assert np.allclose(FH[0], [-0.5 * expect * 0.01, 0, 0], rtol=1e-13)
    assert np.all(FR == 0)
    assert V1[0, 0] == pytest.approx(0.01 + FH[0, 0] / 10.0, rel=1e-15)


def test_zero_relative_velocity_gives_no_force():
    _, d, _ = oracle.corners(np.array([1.3, 2.7, 3.1]))
    U, eN = oracle.stokeslet_fit(d, np.full((8, 3), 1e-3), np.full(3, 1e-3), 0.3)
    assert U == 0.0 and np.all(eN == 0)


# ------------------------------------------------------------ random force (Eqs. 4-5)
@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 11, 13], [123, 456]),
    ([2 ** 64 - 2, 2 ** 64 - 1, 3, 4], [2 ** 64 - 1, 2 ** 63]),
    ([123456789, 42, 0, 0], [3, 0]),
])
def test_philox_matches_numpy(ctr, key):
    """numpy's Philox bit generator is Philox-4x64-10; it increments the counter
    before each block, so its output at counter c is the block function at c+1."""
    ctr = np.array(ctr, np.uint64)
    key = np.array(key, np.uint64)
    ref = np.random.Philox(counter=ctr, key=key).random_raw(4)
    c1 = ctr.copy()
    c1[0] = c1[0] + np.uint64(1)
    if c1[0] == 0:
        c1[1] = c1[1] + np.uint64(1)
    assert np.array_equal(oracle.philox4x64_10(c1, key), ref)


def test_noise_moments_and_uniformity():
    scipy_stats = pytest.importorskip("scipy.stats")
    xi = np.array([oracle.noise_xi(3, n, i) for n in range(400) for i in range(50)])
    assert np.all(np.abs(xi) <= math.sqrt(3))
    assert abs(xi.mean()) < 4 / math.sqrt(xi.size)
    assert xi.var() == pytest.approx(1.0, abs=0.03)
    # uniform on [-sqrt3, sqrt3]
    u = (xi.reshape(-1) / math.sqrt(3) + 1) / 2
    assert scipy_stats.kstest(u, "uniform").pvalue > 1e-3
    # independent components: near-zero correlations
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c - np.eye(3)) < 0.03)


# ------------------------------------------------------------ Langevin update (Eqs. 1-2, 6)
def test_brownian_mode_decays_geometrically():
    """Eq. 6 with dt = 1: V_n = V_0 (1 - gamma/M)^n; the fluid is left untouched."""
    s = oracle.Sim(4, 4, 4, 0.8)
    V0 = np.array([[0.01, -0.02, 0.005]])
    s.add_particles([[1.2, 2.3, 3.4]], V0, [10.0], [0.5], [0.25])
    s.set_params(mode=oracle.BROWNIAN)
    s.step(40)
    _, V, _, _ = s.particles()
    assert np.allclose(V, V0 * (1 - 0.05) ** 40, rtol=1e-13)
    assert np.allclose(s.fhat(), W[:, None, None, None], atol=0)


def test_brownian_mode_ornstein_uhlenbeck_statistics():
    """Discrete OU process: stationary variance (2 gamma kT/M^2)/(1 - a^2) and
    C(k)/C(0) = a^k with a = 1 - gamma/M (the exponential of Eq. 6, Section 3)."""
    M, gamma, kT = 4.0, 1.0, 1e-4
    a = 1 - gamma / M
    n, T = 200, 2000
    s = oracle.Sim(2, 2, 2, 0.8)
    g = np.random.default_rng(0)
    s.add_particles(g.uniform(0, 2, (n, 3)), g.standard_normal((n, 3)) * math.sqrt(kT / M),
                    np.full(n, M), np.full(n, gamma), np.full(n, 0.2))
    s.set_params(kT=kT, seed=9, mode=oracle.BROWNIAN)
    traj = []
    for _ in range(T):
        s.step(1)
        traj.append(s.particles()[1])
    traj = np.array(traj)
    var = (2 * gamma * kT / M ** 2) / (1 - a * a)
    assert traj[200:].var() == pytest.approx(var, rel=0.03)
    cs, cnt = oracle.vacf(traj[200:], 8)
    C = cs / cnt
    assert np.allclose(C / C[0], a ** np.arange(9), atol=0.02)


# ------------------------------------------------------------ VACF estimator (Section 3)
def test_vacf_equals_numpy_correlation():
    g = np.random.default_rng(1)
    T, n, K = 37, 3, 10
    V = g.standard_normal((T, n, 3))
    for stride in (1, 3):
        cs, cnt = oracle.vacf(V, K, stride)
        for k in range(K + 1):
            origins = np.arange(0, T - k, stride)
            ref = sum(np.dot(V[t0, i], V[t0 + k, i]) for t0 in origins for i in range(n))
            assert cs[k] == pytest.approx(ref, rel=1e-13)
            assert cnt[k] == len(origins) * n
        full = sum(np.correlate(V[:, i, c], V[:, i, c], "full")[T - 1:T + K] for i in range(n)
                   for c in range(3))
        if stride == 1:
            assert np.allclose(cs, full, rtol=1e-13)


# ------------------------------------------------------------ coupled step: conservation
@pytest.mark.parametrize("kT,mode", [(0.0, oracle.STOKESLET), (1e-4, oracle.STOKESLET),
                                     (1e-4, oracle.POINTWISE)])
def test_total_momentum_budget(kT, mode):
    """Streaming and BGK conserve momentum, the fluid receives -F_H with weights
    summing to one: total momentum changes only by sum (F_R + F_ext)."""
    L = 10
    s = oracle.Sim(L, L, L, 0.7)
    f0 = wl.perturbed_populations(W, (L, L, L), 1e-3, 2)
    s.set_fhat(f0)
    g = np.random.default_rng(3)
    n = 5
    r0 = g.uniform(0, L, (n, 3))
    V0 = 1e-3 * g.standard_normal((n, 3))
    M = g.uniform(5, 20, n)
    s.add_particles(r0, V0, M, np.full(n, 0.4), np.full(n, 0.3))
    s.set_params(kT=kT, seed=5, mode=mode)
    Fext = 1e-5 * g.standard_normal((n, 3))
    s.set_external(Fext)

    def P():
        fh = s.fhat()
        _, V, _, _ = s.particles()
        return E.T @ fh.reshape(15, -1).sum(1) + (M[:, None] * V).sum(0)

    P0 = P()
    inj = np.zeros(3)
    for _ in range(30):
        s.step(1)
        _, _, FH, FR = s.particles()
        inj += (FR + Fext).sum(0)
        assert np.any(FH != 0)
    assert np.allclose(P() - P0, inj, atol=1e-14)
    assert s.fhat().sum() == pytest.approx(f0.sum(), rel=1e-14)


def test_reaction_force_is_centred_on_the_particle():
    """sum_x F(x) = -F_H and sum_x F(x) (x - r) = 0: trilinear spreading puts the
    reaction force's centre exactly at r_i (Eq. 9)."""
    s = oracle.Sim(8, 8, 8, 0.8)
    r = np.array([[3.3, 4.7, 2.15]])
    s.add_particles(r, [[0.004, -0.003, 0.002]], [10.0], [0.5], [0.26])
    s.set_params()
    s.set_external(None, np.array([1], np.uint8))  # pinned: r stays put
    s.step(1)
    _, _, FH, _ = s.particles()
    F = s.spread_only()
    assert np.allclose(F.reshape(3, -1).sum(1), -FH[0], atol=1e-18)
    zz, yy, xx = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    X = np.stack([xx, yy, zz]).astype(float)
    mom = np.einsum("izyx,jzyx->ij", F, X - r[0][:, None, None, None])
    assert np.allclose(mom, 0, atol=1e-17)


def test_kicked_particle_relaxes_and_fluid_gains_its_momentum():
    """Config of Section 3 (V_R): the particle slows down, F_H opposes V, and in
    a periodic box the final common velocity is M V0 / (M + rho0 L^3)."""
    L, M = 10, 10.0
    s = oracle.Sim(L, L, L, 0.8)
    s.add_particles([[5.5, 5.5, 5.5]], [[0.01, 0, 0]], [M], [0.5], [wl.stokes_radius(0.5, 0.8)])
    s.set_params()
    s.step(1)
    _, V1, FH, _ = s.particles()
    assert FH[0, 0] < 0 and 0 < V1[0, 0] < 0.01
    s.step(1999)
    _, V, _, _ = s.particles()
    assert V[0, 0] == pytest.approx(M * 0.01 / (M + L ** 3), rel=1e-3)
    _, u, _ = s.fields()
    assert np.allclose(u[0], M * 0.01 / (M + L ** 3), rtol=2e-3)


def test_release_response_is_the_kick_response_summed():
    """Fig. 3 / Section 3: for the linear(ised) system the acceleration after a
    force held for T steps is released equals V_R(n+1) - V_R(n+1-T) of a unit
    kick (superposition + time invariance; the FDT relation C = V_R = -A_R in
    its exact discrete form).  Amplitude 1e-8 keeps the system linear."""
    L, T, Tpre, A = 12, 200, 80, 1e-8

    def run(nforce):
        s = oracle.Sim(L, L, L, 0.8)
        s.add_particles([[6.5, 6.5, 6.5]], np.zeros((1, 3)), [10.0], [0.5], [0.26526])
        s.set_params()
        out = []
        for n in range(T):
            s.set_external(np.array([[A, 0, 0]]) if n < nforce else np.zeros((1, 3)))
            s.step(1)
            out.append(s.particles()[1][0, 0])
        return np.array(out)

    kick, rel = run(1), run(Tpre)
    n = np.arange(Tpre, T - 1)
    lhs = rel[n + 1] - rel[n]
    rhs = kick[n + 1] - kick[n + 1 - Tpre]
    assert np.max(np.abs(lhs - rhs)) <= 1e-6 * np.max(np.abs(lhs))


@pytest.mark.slow
def test_long_time_tail_amplitude():
    """C_v(t)/C_v(0) ~ B t^(-3/2), B = M/[12 rho_f (pi nu)^(3/2)] (Section 3, Fig. 2):
    by the FDT the kicked-particle velocity follows the same tail.  64^3 box,
    tau = 0.8, M = 10, gamma = 0.5: B = 4.73; the plateau M V0/(M + L^3) of the
    periodic box is subtracted."""
    L, M, V0 = 64, 10.0, 0.01
    s = oracle.Sim(L, L, L, 0.8)
    s.add_particles([[32.5, 32.5, 32.5]], [[V0, 0, 0]], [M], [0.5], [wl.stokes_radius(0.5, 0.8)])
    s.set_params()
    V = []
    for _ in range(900):
        s.step(1)
        V.append(s.particles()[1][0, 0])
    V = np.array(V) / V0 - M / (M + L ** 3)
    t = np.arange(1, 901)
    nu = 0.1
    B = M / (12 * (math.pi * nu) ** 1.5)
    win = slice(299, 900)
    # sound waves of the periodic images ripple the curve by ~5%: average over t in [300, 900]
    assert np.mean(V[win] * t[win] ** 1.5) == pytest.approx(B, rel=0.05)
    slope = np.polyfit(np.log(t[win]), np.log(V[win]), 1)[0]
    # a power law (an exponential exp(-gamma t / M) of Eq. 6 would be ~1e-9 here);
    # the finite box steepens it slightly beyond -3/2
    assert -1.85 < slope < -1.35


def test_uniform_body_force_adds_its_momentum_every_step():
    """Eqs. 18-19: a uniform force density G on every node adds exactly G of
    momentum per node and step to a uniform fluid, and no mass."""
    nx, ny, nz, n = 6, 5, 4, 7
    o = oracle.Sim(nx, ny, nz, 0.7)
    G = np.array([1.5e-5, -2.0e-5, 0.7e-5])
    o.set_body_force(G)
    o.step(n)
    f = o.fhat()
    E, _ = oracle.d3q15()
    mom = np.einsum("ak,azyx->kzyx", E.astype(float), f)
    assert np.allclose(mom, n * G[:, None, None, None], rtol=0, atol=1e-15)
    assert np.allclose(f.sum(0), 1.0, rtol=0, atol=1e-14)
    o.close()


# ------------------------------------------------------------ point-wise friction (Eq. 7)
def _linear_flow_populations(L, u0, A):
    """Post-collision populations whose streamed (pulled) values at every node x
    away from the periodic seam are f^eq(1, u0 + A x) (Eq. 17): fhat_a(y) =
    f^eq_a(1, u0 + A (y + e_a)), so that f_a(x) = fhat_a(x - e_a)."""
    f = np.empty((15, L, L, L))
    for z in range(L):
        for y in range(L):
            for x in range(L):
                for a in range(15):
                    src = np.array([x, y, z], float) + E[a]
                    f[a, z, y, x] = oracle.feq(1.0, u0 + A @ src)[a]
    return f


def _pointwise_first_step_force(library, r, V, gamma, u0, A, L=10):
    s = oracle.Sim(L, L, L, 0.8, library=library)
    s.set_fhat(_linear_flow_populations(L, u0, A))
    s.add_particles([r], [V], [10.0], [gamma], [0.3])
    s.set_params(mode=oracle.POINTWISE)
    s.step(1)
    FH = s.particles()[2][0]
    s.close()
    return FH


_U0 = np.array([2e-3, -1e-3, 5e-4])
_A = np.array([[3e-4, -2e-4, 1e-4], [1.5e-4, 2.5e-4, -3e-4], [-1e-4, 2e-4, 4e-4]])


@pytest.mark.parametrize("r", [[4.3, 5.6, 3.7], [4.0, 5.0, 3.0], [4.9, 5.05, 3.45]])
def test_pointwise_friction_uses_the_fluid_velocity_at_the_particle(r):
    """Eq. 7, F_H = -gamma (V - u(r_i)), with u(r_i) interpolated from the eight
    corners: in an affine velocity field u(x) = u0 + A x trilinear interpolation is
    exact, so F_H must equal -gamma (V - u0 - A r_i) for any position in the cell
    (a particle on a node sees that node's velocity).  The cell sits away from
    the periodic seam, where the field is affine."""
    r = np.array(r)
    V, gamma = np.array([0.01, -0.004, 0.006]), 0.45
    FH = _pointwise_first_step_force(None, r, V, gamma, _U0, _A)
    expect = -gamma * (V - (_U0 + _A @ r))
    assert np.allclose(FH, expect, rtol=0, atol=1e-13 * np.abs(expect).max())


def test_pointwise_pin_catches_a_swapped_corner_weight(tmp_path):
    """The pin above fails for an oracle copy whose Eq. 7 branch pairs each corner
    velocity with its x-neighbour's weight (a planted mistake, in a copy built
    here; the oracle itself is untouched)."""
    src = open(oracle._SRC).read()
    good = "for (int p = 0; p < 8; ++p) ur += Wp[p] * uN[3 * p + k];"
    assert src.count(good) == 1
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(good, "for (int p = 0; p < 8; ++p) ur += Wp[p ^ 1] * uN[3 * p + k];"))
    so = tmp_path / "libmutant.so"
    import subprocess
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", str(mutant),
                    "-o", str(so), "-lm"], check=True)
    r = np.array([4.3, 5.6, 3.7])
    V, gamma = np.array([0.01, -0.004, 0.006]), 0.45
    FH = _pointwise_first_step_force(oracle.bind(str(so)), r, V, gamma, _U0, _A)
    expect = -gamma * (V - (_U0 + _A @ r))
    assert not np.allclose(FH, expect, rtol=0, atol=1e-13 * np.abs(expect).max())


# ------------------------------------------------------------ MSD (Section 3 dispersion)
def test_msd_equals_the_double_sum_of_velocity_products():
    """With X(t) the running sum of the velocities (Eq. 2 without the wrap), the
    displacement over k steps is the sum of the k velocities after the origin,
    so M(k) = sum_{i,t0} sum_{a,b=1..k} V_i(t0+a).V_i(t0+b) (brute force)."""
    g = np.random.default_rng(7)
    T, n, K = 23, 3, 9
    V = g.standard_normal((T, n, 3))
    X = np.cumsum(V, axis=0) + g.uniform(0, 50, (1, n, 3))
    ms, cnt = oracle.msd(X, K)
    for k in range(K + 1):
        ref = 0.0
        for t0 in range(T - k):
            w = V[t0 + 1:t0 + k + 1]  # [k, n, 3]
            ref += np.einsum("anc,bnc->", w, w)
        assert ms[k] == pytest.approx(ref, rel=1e-12, abs=1e-12)
        assert cnt[k] == n * (T - k)


def test_msd_of_uniform_motion_is_ballistic():
    T, K = 40, 12
    V = np.array([[0.01, -0.02, 0.005], [0.0, 0.003, 0.0]])
    X = np.arange(T)[:, None, None] * V[None] + 3.0
    ms, cnt = oracle.msd(X, K)
    k = np.arange(K + 1)
    assert np.allclose(ms, (T - k) * k ** 2 * (V ** 2).sum(), rtol=1e-12, atol=1e-20)


def test_msd_of_the_ornstein_uhlenbeck_process():
    """Eq. 6 mode: the discrete OU process with C(m) = 3 s2 a^m (s2 the stationary
    variance per component, a = 1 - gamma/M) has
    E|X(t0+k) - X(t0)|^2 = 3 s2 [k + 2 sum_{m<k} (k - m) a^m], which tends to
    6 D k with D = kT/gamma (Einstein): oracle trajectory vs closed form."""
    M, gamma, kT = 4.0, 1.0, 1e-4
    a = 1 - gamma / M
    n, T, K = 300, 1200, 60
    s = oracle.Sim(2, 2, 2, 0.8)
    g = np.random.default_rng(1)
    s.add_particles(g.uniform(0, 2, (n, 3)), g.standard_normal((n, 3)) * math.sqrt(kT / M),
                    np.full(n, M), np.full(n, gamma), np.full(n, 0.2))
    s.set_params(kT=kT, seed=4, mode=oracle.BROWNIAN)
    Vt = []
    for _ in range(T):
        s.step(1)
        Vt.append(s.particles()[1])
    Vt = np.array(Vt)[100:]
    X = np.cumsum(Vt, axis=0)
    ms, cnt = oracle.msd(X, K)
    s2 = (2 * gamma * kT / M ** 2) / (1 - a * a)
    k = np.arange(K + 1)
    expect = np.array([3 * s2 * (kk + 2 * sum((kk - m) * a ** m for m in range(1, kk))) for kk in k])
    assert np.allclose(ms[1:] / cnt[1:], expect[1:], rtol=0.06)
    # long lags: 6 D k with D = kT / gamma, up to the finite-k correction
    D = kT / gamma
    corr = 1 - 2 * a * (1 - a ** K) / (K * (1 - a) * (1 + a))
    assert ms[K] / cnt[K] / (6 * D * K) == pytest.approx(corr, rel=0.06)


@pytest.mark.parametrize("amp", [1e-7, 0.02])
def test_deviation_form_self_check(amp):
    """The oracle run in deviation form (state g = fhat - w_a, moments rho~ - 1
    and u, g^eq = w_a[(rho~ - 1) + 3 u.e + 9/2 (u.e)^2 - 3/2 u.u]; the algebra
    the GPU storage relies on, Eqs. 12-13 and 17 with sum w = 1, sum w e = 0)
    agrees with the full form over 40 coupled steps with noise and an external
    force, to the full form's own FP64 rounding: populations within 8 units in
    the last place of max fhat per step, V within 1e-12 of max |V|, r within
    16 units in the last place of the box size."""
    shape = (9, 10, 12)
    g = np.random.default_rng(1)
    fh = W[:, None, None, None] * (1 + amp * g.uniform(-1, 1, (15,) + shape))
    n, steps = 6, 40
    r = g.uniform(0, 1, (n, 3)) * [12, 10, 9]
    V = g.normal(0, 0.01, (n, 3))
    res = []
    for dev in (False, True):
        s = oracle.Sim(12, 10, 9, 0.7, deviation=dev)
        s.set_fhat(fh)
        s.add_particles(r, V, 6.0, 0.5, 0.2)
        s.set_params(kT=1e-4, seed=3)
        s.set_external(np.full((n, 3), 1e-5))
        s.step(steps)
        rho = s.fields()[0]
        res.append((s.fhat(), *s.particles()[:2], rho))
        s.close()
    (fa, ra, va, rhoa), (fb, rb, vb, rhob) = res
    ulp = 2.0 ** -53
    assert np.abs(fa - fb).max() <= 8 * steps * ulp * np.abs(fa).max()
    assert np.abs(rhoa - rhob).max() <= 16 * steps * ulp * np.abs(rhoa).max()
    assert np.abs(va - vb).max() <= 1e-12 * np.abs(va).max()
    assert np.abs(ra - rb).max() <= 16 * ulp * 12
    # the particles moved the fluid well away from rest: the check is not vacuous
    assert np.abs(fa - W[:, None, None, None]).max() > 1e-4
