"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds the workload recipes (lattice sizes, particle counts, seeds)
and numpy generators of initial states.  It contains none of the method's
arithmetic: it does not stream, collide, fit or integrate anything, and it
imports neither the CUDA binding nor the oracle.

The paper (Section 3) simulates a periodic box of 100^3 nodes with dilute
point particles in a fluid at rest; it publishes no dataset.  The recipes
below keep that structure (periodic box, fluid at rest, uniformly random
particle positions, Maxwellian velocities) at the sizes of the benchmark
configurations.  All quantities are in lattice units dx = dt = rho0 = 1.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import asdict, dataclass, field

import numpy as np

# D3Q15 weights by speed class, used only to build near-equilibrium initial
# populations (rest 2/9, face 1/9, corner 1/72).  The ordering of directions
# is not needed here: callers pass the weight vector of the side they feed.


def stokes_radius(gamma: float, tau: float, rho0: float = 1.0) -> float:
    """Radius for which Stokes' law gamma = 6 pi rho0 nu R holds, nu = (tau - 1/2)/3."""
    nu = (tau - 0.5) / 3.0
    return gamma / (6.0 * math.pi * rho0 * nu)


@dataclass
class ParticleSet:
    r: np.ndarray          # [n, 3] positions in [0, L)
    V: np.ndarray          # [n, 3] velocities
    M: np.ndarray          # [n]
    gamma: np.ndarray      # [n]
    R: np.ndarray          # [n]

    @property
    def n(self) -> int:
        return int(self.r.shape[0])


def uniform_particles(n: int, shape_zyx, M: float, gamma: float, R: float, kT: float,
                      seed_pos: int, seed_vel: int) -> ParticleSet:
    """n particles at uniformly random positions with Maxwellian velocities N(0, kT/M)."""
    nz, ny, nx = shape_zyx
    g = np.random.default_rng(seed_pos)
    r = g.random((n, 3)) * np.array([nx, ny, nz], dtype=np.float64)
    # keep positions strictly inside [0, L) after the float multiply
    r = np.minimum(r, np.nextafter(np.array([nx, ny, nz], dtype=np.float64), 0))
    gv = np.random.default_rng(seed_vel)
    V = gv.standard_normal((n, 3)) * math.sqrt(kT / M) if kT > 0 else np.zeros((n, 3))
    return ParticleSet(r, V, np.full(n, M), np.full(n, gamma), np.full(n, R))


def random_unit_vectors(n: int, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    v = g.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def perturbed_populations(w: np.ndarray, shape_zyx, amp: float, seed: int) -> np.ndarray:
    """f_a(x) = w_a (1 + amp * U(-1, 1)): a non-equilibrium state near rest, [15, nz, ny, nx]."""
    g = np.random.default_rng(seed)
    noise = g.uniform(-1.0, 1.0, (len(w),) + tuple(shape_zyx))
    return w.reshape((-1, 1, 1, 1)) * (1.0 + amp * noise)


@dataclass
class Workload:
    name: str
    shape_zyx: tuple
    tau: float
    n_particles: int
    M: float = 10.0
    gamma: float = 0.5
    kT: float = 0.0
    steps: int = 1000
    seed_pos: int = 1
    seed_vel: int = 2
    seed_noise: int = 3
    vacf_lag: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        nz, ny, nx = self.shape_zyx
        return nx * ny * nz

    @property
    def R(self) -> float:
        return stokes_radius(self.gamma, self.tau)

    def particles(self) -> ParticleSet:
        return uniform_particles(self.n_particles, self.shape_zyx, self.M, self.gamma, self.R,
                                 self.kT, self.seed_pos, self.seed_vel)


# 32^3, one particle at a cell centre, kicked along x, no noise: the single
# particle relaxation run (V_R of Section 3).
RELAXATION_32 = Workload("relaxation_32^3_1p", (32, 32, 32), 0.8, 1, kT=0.0, steps=1000)

# 128^3, 2000 Brownian particles, kT = 1e-4: the VACF run (Fig. 2 structure).
BROWNIAN_128 = Workload("brownian_128^3_2000p", (128, 128, 128), 0.8, 2000, kT=1e-4,
                        steps=20000, vacf_lag=5000)

# 256^3, 16384 particles: storage-precision comparison size.
BROWNIAN_256 = Workload("brownian_256^3_16384p", (256, 256, 256), 0.8, 16384, kT=1e-4,
                        steps=5000)

# 128^3 with 2048 particles (the particle density of the 256^3 case): a small
# case (0.25 GB of populations, still larger than L2) for detailed profiles.
PROFILE_128 = Workload("profile_128^3_2048p", (128, 128, 128), 0.8, 2048, kT=1e-4, steps=100)

# 192^3 with 6912 particles (the bench's particle density): 2 x 212 MB of
# 2-byte populations, larger than L2, for detailed profiles of those kernels.
PROFILE_192 = Workload("profile_192^3_6912p", (192, 192, 192), 0.8, 6912, kT=1e-4, steps=100)

# 64^3 subrun of the 256^3 case at the same number density.
BROWNIAN_64 = Workload("brownian_64^3_256p", (64, 64, 64), 0.8, 256, kT=1e-4, steps=5000)


@dataclass
class Ensemble:
    """Independent periodic boxes (nx, ny, nz, tau) advanced together, n_per_box
    particles in each: the replica ensemble the VACF average of Section 3 is
    taken over, with box size L and viscosity nu varied between replicas."""
    name: str
    boxes: list
    n_per_box: int = 1
    M: float = 10.0
    gamma: float = 0.5
    kT: float = 1e-4
    seed_pos: int = 1
    seed_vel: int = 2
    seed_noise: int = 3

    @property
    def nodes(self) -> int:
        return sum(nx * ny * nz for nx, ny, nz, _ in self.boxes)

    @property
    def n_particles(self) -> int:
        return self.n_per_box * len(self.boxes)

    def particles(self, b: int) -> ParticleSet:
        nx, ny, nz, tau = self.boxes[b]
        R = stokes_radius(self.gamma, tau)
        return uniform_particles(self.n_per_box, (nz, ny, nx), self.M, self.gamma, R, self.kT,
                                 self.seed_pos * 1000 + b, self.seed_vel * 1000 + b)


def _size_classes(classes, taus):
    boxes = []
    for count, L in classes:
        boxes += [(L, L, L, taus[i % len(taus)]) for i in range(count)]
    return boxes


# 48 boxes of 64^3, 16 of 96^3 and 4 of 160^3 (43,122,688 nodes), tau cycling
# over {0.6, 0.8, 1.0} within each size class, one Brownian particle per box.
ENSEMBLE_68 = Ensemble("ensemble_48x64^3+16x96^3+4x160^3_1p",
                       _size_classes([(48, 64), (16, 96), (4, 160)], (0.6, 0.8, 1.0)))


# 64^3, 8 particles kicked to |V0| = 0.01 in seeded random directions, no
# noise, 2000 steps with a checkpoint every 100: the differentiable run
# (gradients of a velocity-relaxation loss by the adjoint).
ADJOINT_64 = Workload("adjoint_64^3_8p", (64, 64, 64), 0.8, 8, kT=0.0, steps=2000,
                      extra={"checkpoint_every": 100, "V0": 0.01, "seed_dir": 4})


def kicked_particles(w: Workload) -> ParticleSet:
    """w.n_particles particles near seeded cell centres (0.35..0.65 into the
    cell, so that the ~0.2-0.3 of relaxation displacement keeps them in their
    cell), velocity V0 along seeded random unit vectors, mass M, friction
    gamma, Stokes radius at w.tau."""
    nz, ny, nx = w.shape_zyx
    g = np.random.default_rng(w.seed_pos)
    cells = np.floor(g.random((w.n_particles, 3)) * np.array([nx, ny, nz]))
    r = cells + g.uniform(0.35, 0.65, (w.n_particles, 3))
    V = random_unit_vectors(w.n_particles, w.extra.get("seed_dir", 4)) * w.extra.get("V0", 0.01)
    n = w.n_particles
    return ParticleSet(r, V, np.full(n, w.M), np.full(n, w.gamma), np.full(n, w.R))


def relaxation_particle(w: Workload, offset=(0.5, 0.5, 0.5), V0=(0.01, 0.0, 0.0)) -> ParticleSet:
    nz, ny, nx = w.shape_zyx
    r = np.array([[nx // 2 + offset[0], ny // 2 + offset[1], nz // 2 + offset[2]]], dtype=np.float64)
    V = np.array([V0], dtype=np.float64)
    return ParticleSet(r, V, np.array([w.M]), np.array([w.gamma]), np.array([w.R]))


# ---------------------------------------------------------------- JSON configs
# A workload as a JSON object: {"kind": "box", "name", "shape_zyx", "tau",
# "n_particles", "M", "gamma", "kT", "steps", "seed_pos", "seed_vel",
# "seed_noise", "vacf_lag", "extra"} or {"kind": "ensemble", "name", "boxes"
# ([nx, ny, nz, tau] each), "n_per_box", "M", "gamma", "kT", seeds}.  The
# files under configs/ hold the five benchmark configurations.

CONFIG_DIR = os.path.join(os.path.dirname(__file__), "configs")


def to_dict(w) -> dict:
    d = asdict(w)
    if isinstance(w, Ensemble):
        d["kind"] = "ensemble"
        d["boxes"] = [list(b) for b in w.boxes]
    else:
        d["kind"] = "box"
        d["shape_zyx"] = list(w.shape_zyx)
    return d


def from_dict(d: dict):
    d = dict(d)
    kind = d.pop("kind", "box")
    if kind == "ensemble":
        d["boxes"] = [tuple(b) for b in d["boxes"]]
        return Ensemble(**d)
    if kind != "box":
        raise ValueError(f"unknown workload kind {kind!r}")
    d["shape_zyx"] = tuple(int(v) for v in d["shape_zyx"])
    return Workload(**d)


def load(path: str):
    """The workload described by a JSON file (see to_dict)."""
    with open(path) as fh:
        return from_dict(json.load(fh))
