"""The physical setting the paper prints (tests/golden/paper_parameters.txt:
the captions of Figs. 1-2 in Section 3 and the closing remarks of Section 2.2),
taken to lattice units, against dimensionless invariants, Stokes' law through
the oracle's fit (Eq. 8) and the validity range the paper states."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_13412_gb300 import experiments as ex
from paper_1909_13412_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def printed():
    """name -> value of every line 'name = value  citation' of the fixture."""
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, rest = line.split("=", 1)
            value, citation = rest.split(None, 1)
            assert citation.startswith("Section"), line
            out[name.strip()] = float(value)
    return out


P = printed()


def test_the_experiments_use_the_printed_setting():
    assert set(ex.PAPER_SI) <= set(P)
    for k, v in ex.PAPER_SI.items():
        assert v == P[k], k


def test_lattice_units_of_the_printed_setting():
    """dx = dt = rho0 = 1: L = box/dx, nu dt/dx^2, U dt/dx, R/dx, M/(rho0 dx^3)."""
    lu = ex.lattice_units(**P)
    assert lu["L"] == pytest.approx(100.0, rel=1e-14)
    assert lu["nu"] == pytest.approx(0.0178, rel=1e-13)
    assert lu["tau"] == pytest.approx(0.5534, rel=1e-13)  # nu = (tau - 1/2)/3, Eq. 16
    assert ex.nu_of(lu["tau"]) == pytest.approx(lu["nu"], rel=1e-12)
    assert lu["U"] == pytest.approx(1e-4, rel=1e-13)
    assert lu["R"] == pytest.approx(1.0, rel=1e-14)
    assert lu["M"] == pytest.approx(16.0, rel=1e-13)
    # the dimensionless groups do not depend on the units: the Reynolds number
    # U R / nu of Section 3 and the mass ratio M / (rho0 R^3)
    assert lu["U"] * lu["R"] / lu["nu"] == pytest.approx(P["U"] * P["R"] / P["nu"], rel=1e-13)
    assert lu["M"] / lu["R"] ** 3 == pytest.approx(P["M"] / (P["rho0"] * P["R"] ** 3), rel=1e-13)
    # low Mach number: the flow is far below the lattice sound speed 1/sqrt(3)
    assert lu["U"] * math.sqrt(3.0) < 1e-3


def _stokes_field(d, e, R):
    """Uniform stream e minus the Stokeslet of a sphere of radius R (Oseen tensor)."""
    out = []
    for dp in d:
        r = np.linalg.norm(dp)
        G = np.eye(3) / r + np.outer(dp, dp) / r ** 3
        out.append(e - 0.75 * R * G @ e)
    return np.array(out)


@pytest.mark.parametrize("pos,e", [((50.5, 50.5, 50.5), (0.36, 0.48, -0.8)),
                                   ((3.5, 97.5, 12.5), (0.0, -0.6, 0.8))])
def test_stokes_law_of_the_fit_in_si_units(pos, e):
    """Fig. 1: in an exact Stokes flow of speed U past the printed sphere at a
    cell centre, the fit of Eq. 8 recovers the flow at infinity, and
    F_H = 6 pi rho0 nu R U_inf e^N in lattice units, brought back to SI (force
    unit rho0 dx^4 / dt^2), is the printed Stokes law 6 pi eta R U, eta =
    rho0 nu.  With R = dx every corner (at sqrt(3)/2 dx) lies inside the
    sphere, where the Stokeslet term outweighs the stream: the mean of the
    corner velocities, and with it e^N, points against the flow, and the fit
    returns U_inf = -U, so that U_inf e^N is still the flow at infinity."""
    lu = ex.lattice_units(**P)
    _, d, _ = oracle.corners(np.array(pos))
    e = np.array(e)
    w = lu["U"] * _stokes_field(d, e, lu["R"])
    # at a cell centre the corners' mean of the Stokes flow is U e (1 - 2R/sqrt(3))
    # (mean of I/r + d d^T/r^3 over the corners: (2/sqrt(3) + 1/(4 r^3)) I with
    # r = sqrt(3)/2): zero at R = sqrt(3)/2, reversed beyond
    assert np.allclose(w.mean(axis=0), lu["U"] * e * (1.0 - 2.0 * lu["R"] / math.sqrt(3.0)),
                       rtol=0, atol=1e-15)
    U, eN = oracle.stokeslet_fit(d, w, np.zeros(3), lu["R"])
    assert np.allclose(eN, -e, atol=1e-13)
    assert U == pytest.approx(-lu["U"], rel=1e-12)
    F_lattice = 6.0 * math.pi * lu["nu"] * lu["R"] * U * eN
    F_si = F_lattice * P["rho0"] * P["dx"] ** 4 / P["dt"] ** 2
    stokes = 6.0 * math.pi * (P["rho0"] * P["nu"]) * P["R"] * P["U"] * e
    assert np.allclose(F_si, stokes, rtol=1e-12, atol=1e-12 * np.abs(stokes).max())


def test_tail_amplitude_in_lattice_units():
    """Fig. 2: B = M / [12 rho_f (pi nu)^(3/2)] has the units of time^(3/2);
    in lattice units it is the SI value over dt^(3/2), whatever the other
    scales, and the experiments' B (from tau) is that value."""
    lu = ex.lattice_units(**P)
    B_si = P["M"] / (12.0 * P["rho0"] * (math.pi * P["nu"]) ** 1.5)
    B_lattice = lu["M"] / (12.0 * (math.pi * lu["nu"]) ** 1.5)
    assert B_lattice == pytest.approx(B_si / P["dt"] ** 1.5, rel=1e-12)
    assert lu["M"] / (12.0 * (math.pi * ex.nu_of(lu["tau"])) ** 1.5) == pytest.approx(B_lattice, rel=1e-12)


def _phi(n, R, nodes):
    return n * 4.0 / 3.0 * math.pi * R ** 3 / nodes


def test_workloads_lie_in_the_range_the_method_was_checked_for():
    """Section 2.2: volume fraction below 0.1 and R up to about sqrt(3) dx.  The
    Fig. 2 suspension itself, every synthetic workload and every box of the
    replica ensemble are inside both."""
    assert P["R_max_dx"] == pytest.approx(math.sqrt(3.0), rel=1e-15)
    lu = ex.lattice_units(**P)
    assert _phi(P["n_particles"], lu["R"], lu["L"] ** 3) < P["phi_max"]
    assert lu["R"] < P["R_max_dx"]
    for w in (wl.RELAXATION_32, wl.BROWNIAN_64, wl.BROWNIAN_128, wl.BROWNIAN_256, wl.PROFILE_128,
              wl.PROFILE_192, wl.ADJOINT_64):
        assert w.R < P["R_max_dx"], w.name
        assert _phi(w.n_particles, w.R, w.nodes) < P["phi_max"], w.name
    e = wl.ENSEMBLE_68
    for nx, ny, nz, tau in e.boxes:
        R = wl.stokes_radius(e.gamma, tau)
        assert R < P["R_max_dx"]
        assert _phi(e.n_per_box, R, nx * ny * nz) < P["phi_max"]
