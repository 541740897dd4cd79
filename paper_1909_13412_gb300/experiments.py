"""The paper's numerical experiments (Section 3) run on the GPU through the C ABI.

  * ``pinned_sphere_drag`` -- Fig. 1: the hydrodynamic force on a sphere held
    at rest in a uniform flow U, for the present method (Stokeslet fit, Eq. 8)
    and the point-wise friction model (Eq. 7), against Stokes' law
    F = 6 pi eta R U.  The box is periodic, so the flow is that past a simple
    cubic array of spheres: Hasimoto's (1959) correction of Stokes' law for
    such an array, F = 6 pi eta R U / K(c), K = 1 - 1.7601 c^(1/3) + c
    - 1.5593 c^2, c = (4 pi / 3)(R / L)^3, is reported beside it.  The fluid
    starts at the equilibrium of velocity U; a uniform body force equal to the
    drag per node (fed back from the measured F_H) keeps the mean flow at U.
  * ``kick_and_release`` -- Fig. 3: the velocity V_R(t) of a particle kicked
    from rest and the acceleration A_R(t) = V(t + 1) - V(t) of a particle
    released after a constant force was held for ``t_hold`` steps.
  * ``brownian_vacf`` -- Fig. 2 / Fig. 3: the normalised VACF C_v(t)/C_v(0)
    of Brownian particles (the library's all-origins estimator).
  * ``tail_amplitude`` -- the long-time tail C_v(t)/C_v(0) ~ B t^(-3/2),
    B = M / [12 rho0 (pi nu)^(3/2)], measured on the kicked particle.
  * ``brownian_run`` / ``config2`` -- the Brownian suspension at its stated
    size and length (128^3, 2000 particles, kT = 1e-4, 2 x 10^4 steps, VACF
    and MSD to lag 5000), in independent realisations: particle updates per
    second, the log-log slope and amplitude of the VACF tail over a window
    with their spread over the realisations, and the diffusion coefficient
    from the MSD against the Green-Kubo integral of the VACF.

Every step of every run is the library's CUDA path; this module only sets up
inputs, reads results and does the bookkeeping of each experiment.  Run as
``python -m paper_1909_13412_gb300.experiments fig1|fig3|tail|config2`` for the
tables (``config2 --config FILE.json`` for another workload file).
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import lbp


def nu_of(tau):
    """Kinematic viscosity of the BGK fluid, Eq. 16 (lattice units)."""
    return (tau - 0.5) / 3.0


# The physical setting of Figs. 1-2 (Section 3, the figure captions), SI units:
# box edge, grid interval, time step, kinematic viscosity and density of the
# fluid, the flow speed of Fig. 1, and the particles of Fig. 2.
PAPER_SI = {"box": 500e-9, "dx": 5e-9, "dt": 0.5e-12, "nu": 0.89e-6, "rho0": 1.0e3, "U": 1.0,
            "n_particles": 500, "R": 5e-9, "M": 2e-21}


def lattice_units(box, dx, dt, nu, rho0, U, R, M, **_):
    """The setting in lattice units (dx = dt = rho0 = 1): box edge L in nodes,
    tau from nu = (tau - 1/2)/3 (Eq. 16), flow speed, radius and mass."""
    nu_l = nu * dt / dx ** 2
    return {"L": box / dx, "nu": nu_l, "tau": 0.5 + 3.0 * nu_l, "U": U * dt / dx, "R": R / dx,
            "M": M / (rho0 * dx ** 3)}


def hasimoto_factor(R, L):
    """K(c) of Hasimoto (1959) for a simple cubic array of spheres of radius R
    and period L: the drag is 6 pi eta R U / K."""
    c = 4.0 * math.pi / 3.0 * (R / L) ** 3
    return 1.0 - 1.7601 * c ** (1.0 / 3.0) + c - 1.5593 * c * c


def pinned_sphere_drag(L, tau, U, R, mode=lbp.LBP_STOKESLET, steps=20000, hold_every=20,
                       offset=(0.5, 0.5, 0.5), average_last=0.1):
    """Steady drag F_H (x component) on a pinned particle of radius R in a
    periodic L^3 box whose fluid moves at mean velocity U along x."""
    N = L ** 3
    h = lbp.lbp_create(L, L, L, tau)
    try:
        lbp.lbp_set_use_graphs(h, False)  # the body force changes every hold_every steps
        u = np.zeros((3, N))
        u[0] = U
        lbp.lbp_set_fluid(h, None, u)
        eta = nu_of(tau)  # rho0 = 1
        gamma = 6.0 * math.pi * eta * R
        r = np.array([[L // 2 + offset[0], L // 2 + offset[1], L // 2 + offset[2]]])
        lbp.lbp_particles_add(h, r, np.zeros((1, 3)), np.array([1.0]), np.array([gamma]), np.array([R]))
        lbp.lbp_particles_set_params(h, kT=0.0, seed=0, mode=mode)
        lbp.lbp_particles_set_external_force(h, None, np.array([1], np.uint8))
        F = np.zeros((1, 3))
        hist = []
        for _ in range(max(1, steps // hold_every)):
            lbp.lbp_step(h, hold_every)
            lbp.lbp_particles_read(h, f_h=F)
            # the fluid lost F_H per step to the particle: give it back uniformly
            lbp.lbp_set_body_force(h, F[0] / N)
            hist.append(F[0, 0])
        lbp.lbp_check(h)
    finally:
        lbp.lbp_destroy(h)
    hist = np.array(hist)
    k = max(1, int(len(hist) * average_last))
    F_ss = float(np.mean(hist[-k:]))
    stokes = 6.0 * math.pi * nu_of(tau) * R * U
    return {"R": R, "F_H": F_ss, "stokes": stokes, "F_over_stokes": F_ss / stokes,
            "hasimoto": stokes / hasimoto_factor(R, L),
            "F_over_hasimoto": F_ss / (stokes / hasimoto_factor(R, L)),
            "drift_last": float(abs(hist[-1] - hist[-k]) / abs(F_ss)) if F_ss else 0.0,
            "steps": len(hist) * hold_every}


def kick_and_release(L, tau, M, gamma, R, amplitude, T, t_hold, position=None):
    """V_R(t): velocity after a kick V0 = amplitude / M from rest (one step of
    external force `amplitude`); A_R(t) = V(t + 1) - V(t) after a force
    `amplitude` held for t_hold steps is released.  Both [T] arrays (x)."""
    pos = np.array([position or [L // 2 + 0.5] * 3], dtype=np.float64)

    def run(n_force):
        h = lbp.lbp_create(L, L, L, tau)
        try:
            lbp.lbp_set_use_graphs(h, False)
            lbp.lbp_particles_add(h, pos, np.zeros((1, 3)), np.array([M]), np.array([gamma]), np.array([R]))
            lbp.lbp_particles_set_params(h, kT=0.0, seed=0)
            V = np.zeros((1, 3))
            out = np.empty(T + n_force)
            force = np.array([[amplitude, 0.0, 0.0]])
            lbp.lbp_particles_set_external_force(h, force)
            for n in range(T + n_force):
                if n == n_force:
                    lbp.lbp_particles_set_external_force(h, np.zeros((1, 3)))
                lbp.lbp_step(h, 1)
                lbp.lbp_particles_read(h, v=V)
                out[n] = V[0, 0]
            return out
        finally:
            lbp.lbp_destroy(h)

    kick = run(1)[:T]                 # V after steps 1..T (force acted during step 0)
    held = run(t_hold)
    rel = held[t_hold - 1:]           # V at release (index 0) and after
    A_R = rel[1:T + 1] - rel[:T]
    return kick, A_R


def brownian_vacf(L, tau, n, M, gamma, kT, steps, max_lag, mode=lbp.LBP_STOKESLET, seed=1):
    """Normalised VACF of n Brownian particles (uniform positions, Maxwellian
    start) after `steps` steps: C(k)/C(0), k = 0..max_lag."""
    from . import workloads as wl
    ps = wl.uniform_particles(n, (L, L, L), M, gamma, wl.stokes_radius(gamma, tau), kT, seed, seed + 1)
    h = lbp.lbp_create(L, L, L, tau)
    try:
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=seed + 2, mode=mode)
        lbp.lbp_vacf_configure(h, max_lag)
        lbp.lbp_step(h, steps)
        cs = np.empty(max_lag + 1)
        cnt = np.empty(max_lag + 1, np.int64)
        lbp.lbp_vacf_read(h, cs, cnt)
        lbp.lbp_check(h)
    finally:
        lbp.lbp_destroy(h)
    C = cs / np.maximum(cnt, 1)
    return C / C[0]


def tail_amplitude(L, tau, M, gamma, T, window, V0=0.01):
    """Kick a particle (V0 along x) in a fluid at rest and fit the tail
    (V(t)/V0 - plateau) t^(3/2) over `window` = (t0, t1); the plateau
    M V0/(M + L^3) of the periodic box is removed.  Returns (measured B, B of
    M / [12 rho0 (pi nu)^(3/2)], slope of log V vs log t)."""
    h = lbp.lbp_create(L, L, L, tau)
    try:
        R = gamma / (6.0 * math.pi * nu_of(tau))
        lbp.lbp_particles_add(h, np.array([[L // 2 + 0.5] * 3]), np.array([[V0, 0.0, 0.0]]),
                              np.array([M]), np.array([gamma]), np.array([R]))
        lbp.lbp_particles_set_params(h, kT=0.0, seed=0)
        vt = np.empty((T, 1, 3))
        lbp.lbp_adjoint_record(h, T, T, vt, None)  # one recording run = the whole trajectory
    finally:
        lbp.lbp_destroy(h)
    V = vt[:, 0, 0] / V0 - M / (M + L ** 3)
    t = np.arange(1, T + 1)
    t0, t1 = window
    sl = slice(t0 - 1, t1)
    B = float(np.mean(V[sl] * t[sl] ** 1.5))
    slope = float(np.polyfit(np.log(t[sl]), np.log(V[sl]), 1)[0])
    return B, M / (12.0 * (math.pi * nu_of(tau)) ** 1.5), slope


def brownian_run(L, tau, n, M, gamma, kT, steps, max_lag, seed):
    """One realisation of a Brownian suspension: n particles at uniform random
    positions with Maxwellian velocities, `steps` steps, VACF and MSD to
    `max_lag`.  Returns (C(k)/C(0), MSD(k) per pair, C(0) per pair, seconds of
    stepping, measured on the device)."""
    import time
    from . import workloads as wl
    ps = wl.uniform_particles(n, (L, L, L), M, gamma, wl.stokes_radius(gamma, tau), kT, seed, seed + 1)
    h = lbp.lbp_create(L, L, L, tau)
    try:
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=seed + 2)
        lbp.lbp_step(h, 2)
        lbp.lbp_autotune(h, 5)
        lbp.lbp_vacf_configure(h, max_lag)
        cs = np.empty(max_lag + 1)
        cnt = np.empty(max_lag + 1, np.int64)
        ms = np.empty(max_lag + 1)
        lbp.lbp_vacf_read(h, cs, cnt)  # waits for the set-up
        t0 = time.perf_counter()
        lbp.lbp_step(h, steps)
        lbp.lbp_vacf_read(h, cs, cnt)  # host read: waits for every step and block
        secs = time.perf_counter() - t0
        lbp.lbp_msd_read(h, ms, cnt)
        lbp.lbp_check(h)
    finally:
        lbp.lbp_destroy(h)
    C = cs / cnt
    return C / C[0], ms / cnt, float(C[0]), secs


def config2_statistics(runs, window, M, tau):
    """Tail statistics of independent realisations (lists of C/C(0) and MSD
    arrays): per realisation the log-log slope of C/C(0) over `window` and the
    amplitude B = mean over the window of C/C(0) t^(3/2); reported as the
    mean and the standard error over realisations.  D from the MSD's slope
    over the last half of the lags (per component: MSD / 6 per step) against
    the Green-Kubo integral of the VACF over the same lags."""
    t0, t1 = window
    t = np.arange(t0, t1 + 1)
    slopes, amps, d_msd, d_gk = [], [], [], []
    for C, msd, c0 in runs:
        y = C[t0:t1 + 1]
        slopes.append(float(np.polyfit(np.log(t), np.log(np.abs(y)), 1)[0]))
        amps.append(float(np.mean(y * t ** 1.5)))
        K = len(msd) - 1
        k = np.arange(K // 2, K + 1)
        d_msd.append(float(np.polyfit(k, msd[K // 2:], 1)[0] / 6.0))
        # discrete Green-Kubo: MSD(k)/k -> C(0) + 2 sum_{m>=1} C(m) (per pair), over 6
        d_gk.append(float(c0 * (1.0 + 2.0 * C[1:K // 2].sum()) / 6.0))
    n = len(runs)
    se = lambda v: float(np.std(v, ddof=1) / math.sqrt(n)) if n > 1 else float("nan")
    return {"window": [t0, t1], "realisations": n,
            "slope": float(np.mean(slopes)), "slope_se": se(slopes),
            "B": float(np.mean(amps)), "B_se": se(amps),
            "B_paper": M / (12.0 * (math.pi * nu_of(tau)) ** 1.5),
            "D_msd": float(np.mean(d_msd)), "D_msd_se": se(d_msd),
            "D_green_kubo": float(np.mean(d_gk)), "D_green_kubo_se": se(d_gk)}


def ensemble_groups(boxes):
    """Box indices of each (L, tau) group of a replica ensemble ((nx, ny, nz, tau)
    per box, cubic), in order of first appearance: the VACF is averaged within a
    group, since averaging across tau would mix viscosities (Section 3 takes the
    VACF over replicas of one suspension)."""
    groups = {}
    for b, (nx, ny, nz, tau) in enumerate(boxes):
        groups.setdefault((nx, tau), []).append(b)
    return groups


def ensemble_run(w, steps, max_lag, seed, mode=lbp.LBP_STOKESLET):
    """The batched ensemble `w` (one handle, one particle launch and one lattice
    launch per step over all boxes) for `steps` steps with the per-particle VACF
    to `max_lag`.  Returns the per-particle sums [n, K + 1], the pair counts
    per lag [K + 1] and the seconds of stepping (device-waited).  `mode`: the
    coupling (Eq. 8 by default; Eq. 6 leaves the fluid out)."""
    import time
    h = lbp.lbp_create_batch(w.boxes)
    try:
        for b in range(len(w.boxes)):
            pb = w.particles(b)
            lbp.lbp_particles_add_to(h, b, pb.r, pb.V, pb.M, pb.gamma, pb.R)
        lbp.lbp_particles_set_params(h, kT=w.kT, seed=seed, mode=mode)
        lbp.lbp_step(h, 2)
        lbp.lbp_autotune(h, 5)
        lbp.lbp_vacf_configure_ex(h, max_lag, 1)
        cs = np.empty((w.n_particles, max_lag + 1))
        cnt = np.empty(max_lag + 1, np.int64)
        lbp.lbp_vacf_read_per_particle(h, cs, cnt)  # waits for the set-up
        t0 = time.perf_counter()
        lbp.lbp_step(h, steps)
        lbp.lbp_vacf_read_per_particle(h, cs, cnt)  # host read: waits for every step and block
        secs = time.perf_counter() - t0
        lbp.lbp_check(h)
    finally:
        lbp.lbp_destroy(h)
    return cs, cnt, secs


def ensemble_statistics(w, cs, cnt, window, lags=(1, 10, 50, 100, 200, 400, 1000)):
    """Per (L, tau) group: the group's VACF C(k) = sum over its particles of the
    per-particle sums / (particles x pairs per lag), C(k)/C(0) at `lags`, C(0)
    per pair (not 3 kT/M with the athermal fluid: the particle drags it along),
    and the tail amplitude B = mean over `window`
    of C/C(0) t^(3/2) with the standard error over the group's particles (each
    particle's own C_i/C_i(0)), beside M/[12 rho (pi nu)^(3/2)] at the group's tau."""
    t0, t1 = window
    t = np.arange(t0, t1 + 1)
    K = cs.shape[1] - 1
    per = w.n_per_box
    out = []
    for (L, tau), boxes in ensemble_groups(w.boxes).items():
        rows = [b * per + q for b in boxes for q in range(per)]
        C = cs[rows].sum(axis=0) / (len(rows) * cnt)
        Ci = cs[rows] / cnt
        amps = [float(np.mean(c[t0:t1 + 1] / c[0] * t ** 1.5)) for c in Ci]
        n = len(amps)
        out.append({"L": int(L), "tau": float(tau), "boxes": len(boxes), "particles": n,
                    "C0": float(C[0]),
                    "C_over_C0": {str(k): float(C[k] / C[0]) for k in lags if k <= K},
                    "B": float(np.mean(C[t0:t1 + 1] / C[0] * t ** 1.5)),
                    "B_se": float(np.std(amps, ddof=1) / math.sqrt(n)) if n > 1 else float("nan"),
                    "B_paper": w.M / (12.0 * (math.pi * nu_of(tau)) ** 1.5)})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("experiment", choices=["fig1", "fig3", "tail", "config2", "config4"])
    ap.add_argument("--realisations", type=int, default=4)
    ap.add_argument("--window", type=int, nargs=2, default=[100, 400])
    ap.add_argument("--config", default=None,
                    help="config2: a workload JSON file (cubic box, vacf_lag > 0) instead of "
                         "configs/config2_brownian_128.json")
    ap.add_argument("--paper", action="store_true",
                    help="fig1 at the paper's parameters (100^3 box, nu = 0.0178, U = 1e-4)")
    a = ap.parse_args(argv)
    if a.experiment == "fig1":
        if a.paper:
            # Section 3 / Fig. 1: box 500 nm, dx = 5 nm, dt = 0.5 ps, nu = 0.89e-6 m^2/s,
            # U = 1 m/s -> L = 100, nu = 0.0178 (tau = 0.5534), U = 1e-4 (lattice units)
            lu = lattice_units(**PAPER_SI)
            L, tau, U, steps = int(round(lu["L"])), lu["tau"], lu["U"], 120000
        else:
            L, tau, U, steps = 40, 0.8, 1e-4, 8000
        rows = []
        for R in (0.2, 0.4, 0.6, 0.8, 1.0, 1.2, 1.4):
            for mode, name in ((lbp.LBP_STOKESLET, "present"), (lbp.LBP_POINTWISE, "pointwise")):
                d = pinned_sphere_drag(L, tau, U, R, mode, steps)
                d.update({"model": name, "L": L, "tau": tau, "U": U})
                rows.append(d)
                print(json.dumps(d), flush=True)
    elif a.experiment == "fig3":
        kick, A_R = kick_and_release(32, 0.8, 10.0, 0.5, 0.5 / (6 * math.pi * 0.1), 1e-8, 400, 2000)
        C = brownian_vacf(64, 0.8, 256, 10.0, 0.5, 1e-4, 20000, 400)
        print(json.dumps({"t": [1, 5, 10, 20, 50, 100, 200, 400],
                          "V_R": [float(kick[t - 1] / kick[0]) for t in (1, 5, 10, 20, 50, 100, 200, 400)],
                          "A_R": [float(A_R[t - 1] / A_R[0]) for t in (1, 5, 10, 20, 50, 100, 200, 400)],
                          "C_v": [float(C[t - 1] / C[0]) for t in (1, 5, 10, 20, 50, 100, 200, 400)]}))
    elif a.experiment == "config2":
        from . import workloads as wl
        w = wl.load(a.config) if a.config else wl.BROWNIAN_128
        if len(set(w.shape_zyx)) != 1 or w.vacf_lag <= 0:
            raise SystemExit("config2 needs a cubic box and vacf_lag > 0")
        L, tau, n, kT = w.shape_zyx[0], w.tau, w.n_particles, w.kT
        runs, secs = [], []
        for r in range(a.realisations):
            C, msd, c0, sec = brownian_run(L, tau, n, w.M, w.gamma, kT, w.steps, w.vacf_lag, 100 + 10 * r)
            runs.append((C, msd, c0))
            secs.append(sec)
        out = config2_statistics(runs, tuple(a.window), w.M, tau)
        out.update({"workload": w.name, "steps": w.steps, "max_lag": w.vacf_lag,
                    "particle_updates_per_s": n * w.steps / float(np.mean(secs)),
                    "mlups": L ** 3 * w.steps / float(np.mean(secs)) / 1e6,
                    "C_over_C0": {str(t): float(np.mean([c[0][t] for c in runs])) for t in
                                  (1, 10, 50, 100, 200, 400, 1000)}})
        print(json.dumps(out))
    elif a.experiment == "config4":
        from . import workloads as wl
        w = wl.load(a.config) if a.config else wl.ENSEMBLE_68
        steps, max_lag = 10000, 5000
        cs, cnt, secs = ensemble_run(w, steps, max_lag, w.seed_noise)
        print(json.dumps({"workload": w.name, "steps": steps, "max_lag": max_lag,
                          "mlups": w.nodes * steps / secs / 1e6,
                          "particle_updates_per_s": w.n_particles * steps / secs,
                          "window": list(a.window),
                          "groups": ensemble_statistics(w, cs, cnt, tuple(a.window))}))
    else:
        B, B_th, slope = tail_amplitude(128, 0.8, 10.0, 0.5, 3000, (600, 2000))
        print(json.dumps({"B_measured": B, "B_theory": B_th, "slope": slope}))


if __name__ == "__main__":
    main()
