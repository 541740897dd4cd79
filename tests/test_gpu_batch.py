"""Batched ensembles: several independent periodic boxes in one handle.

A batch (lbp_create_batch) lays the boxes' nodes one after another in the same
population planes and advances them all with one lattice launch and one
particle launch per step.  The boxes do not interact, so every box of a batch
must evolve exactly as the same box simulated alone:

  * populations, fields and particle states bitwise equal to separate
    single-box handles, for every storage precision, when no random force is
    drawn (kT = 0);
  * with kT > 0 the random force of particle i uses the Philox counter
    (step, i) with i its index in the handle, so box 0 (particles 0..n0-1 in
    both) is still bitwise equal to its single-box run;
  * per-particle VACF sums add up to the ensemble VACF and match the
    trajectory read back step by step.
"""
import numpy as np
import pytest

from paper_1909_13412_gb300 import lbp
from paper_1909_13412_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 15
# D3Q15 weights in the library's direction order (rest, 6 faces, 8 corners)
W = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)

# uneven boxes: ragged x tails, x wider than one 128-node segment, odd row counts
BOXES = [(20, 18, 16, 0.8), (33, 7, 12, 0.6), (130, 5, 4, 1.0), (8, 8, 8, 0.7)]
NPART = [7, 3, 5, 0]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1909_13412_gb300 import build as lbp_build
    lbp_build.build()
    lbp.load()
    torch.cuda.set_device(0)


def box_state(b, box):
    nx, ny, nz, tau = box
    f = wl.perturbed_populations(W, (nz, ny, nx), 0.02, 100 + b)
    ps = wl.uniform_particles(NPART[b], (nz, ny, nx), 6.0, 0.5, 0.0, 1e-4, 10 + b, 20 + b)
    ps.R = np.full(ps.n, wl.stokes_radius(0.5, tau))
    ps.V = np.random.default_rng(30 + b).normal(0.0, 0.01, (ps.n, 3))
    return f, ps


def run_single(b, box, prec, steps, kT, graphs):
    nx, ny, nz, tau = box
    f, ps = box_state(b, box)
    h = lbp.lbp_create(nx, ny, nz, tau, precision=prec)
    lbp.lbp_set_use_graphs(h, graphs)
    lbp.lbp_set_populations(h, f)
    if ps.n:
        lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
        lbp.lbp_particles_set_params(h, kT=kT, seed=5)
    lbp.lbp_step(h, steps)
    lbp.lbp_check(h)
    fo = np.empty((Q, nz, ny, nx))
    lbp.lbp_read_populations(h, fo)
    parts = [np.empty((ps.n, 3)) for _ in range(4)]
    if ps.n:
        lbp.lbp_particles_read(h, *parts)
    lbp.lbp_destroy(h)
    return fo, parts


def make_batch(prec, kT, graphs):
    h = lbp.lbp_create_batch(BOXES, precision=prec)
    lbp.lbp_set_use_graphs(h, graphs)
    fall = np.concatenate([box_state(b, bx)[0].reshape(Q, -1) for b, bx in enumerate(BOXES)], axis=1)
    lbp.lbp_set_populations(h, fall)
    for b, bx in enumerate(BOXES):
        _, ps = box_state(b, bx)
        if ps.n:
            lbp.lbp_particles_add_to(h, b, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=kT, seed=5)
    return h


def read_batch(h):
    f = np.empty((Q, h.N))
    lbp.lbp_read_populations(h, f)
    n = lbp.lbp_particles_count(h)
    parts = [np.empty((n, 3)) for _ in range(4)]
    lbp.lbp_particles_read(h, *parts)
    return f, parts


def test_replica_info_and_offsets():
    h = lbp.lbp_create_batch(BOXES)
    assert lbp.lbp_replica_count(h) == len(BOXES)
    off = 0
    for b, (nx, ny, nz, tau) in enumerate(BOXES):
        dims, t, o = lbp.lbp_replica_info(h, b)
        assert dims == (nx, ny, nz) and t == tau and o == off
        off += nx * ny * nz
    assert h.N == off
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_replica_info(h, len(BOXES))
    assert ei.value.status == lbp.LBP_EINVAL
    lbp.lbp_destroy(h)


@pytest.mark.parametrize("prec", [lbp.LBP_F32, lbp.LBP_BF16, lbp.LBP_F16])
@pytest.mark.parametrize("graphs", [True, False])
def test_batch_bitwise_equals_separate_boxes(prec, graphs):
    steps = 40
    h = make_batch(prec, 0.0, graphs)
    lbp.lbp_step(h, steps)
    lbp.lbp_check(h)
    f, parts = read_batch(h)
    lbp.lbp_destroy(h)
    off, p0 = 0, 0
    for b, bx in enumerate(BOXES):
        nx, ny, nz, _ = bx
        fs, ps = run_single(b, bx, prec, steps, 0.0, graphs)
        n = nx * ny * nz
        assert np.array_equal(f[:, off:off + n].reshape(Q, nz, ny, nx), fs), b
        for k in range(4):
            assert np.array_equal(parts[k][p0:p0 + NPART[b]], ps[k]), (b, k)
        off += n
        p0 += NPART[b]


def test_batch_box0_with_noise_bitwise():
    steps = 30
    h = make_batch(lbp.LBP_F32, 1e-4, True)
    lbp.lbp_step(h, steps)
    f, parts = read_batch(h)
    lbp.lbp_destroy(h)
    nx, ny, nz, _ = BOXES[0]
    fs, ps = run_single(0, BOXES[0], lbp.LBP_F32, steps, 1e-4, True)
    assert np.array_equal(f[:, :nx * ny * nz].reshape(Q, nz, ny, nx), fs)
    for k in range(4):
        assert np.array_equal(parts[k][:NPART[0]], ps[k]), k
    # the random force did act: the other boxes differ from their kT = 0 run
    fs1, ps1 = run_single(1, BOXES[1], lbp.LBP_F32, steps, 0.0, True)
    assert not np.array_equal(parts[1][NPART[0]:NPART[0] + NPART[1]], ps1[1])


def test_batch_fields_are_the_boxes_fields():
    h = make_batch(lbp.LBP_F32, 0.0, True)
    lbp.lbp_step(h, 5)
    rho = np.empty(h.N)
    u = np.empty((3, h.N))
    lbp.lbp_read_fields(h, rho, u)
    f = np.empty((Q, h.N))
    lbp.lbp_read_populations(h, f)
    lbp.lbp_destroy(h)
    off = 0
    for b, (nx, ny, nz, tau) in enumerate(BOXES):
        n = nx * ny * nz
        hs = lbp.lbp_create(nx, ny, nz, tau)
        lbp.lbp_set_populations(hs, np.ascontiguousarray(f[:, off:off + n]))
        rs = np.empty(n)
        us = np.empty((3, n))
        lbp.lbp_read_fields(hs, rs, us)
        lbp.lbp_destroy(hs)
        assert np.array_equal(rho[off:off + n], rs), b
        assert np.array_equal(u[:, off:off + n], us), b
        off += n


def test_particles_add_to_validates_against_its_box():
    h = lbp.lbp_create_batch(BOXES)
    one = lambda x: np.array([x], dtype=np.float64)
    # inside box 2 (130 x 5 x 4) but outside box 1 (33 x 7 x 12) along x
    r = np.array([[100.0, 1.0, 1.0]])
    V = np.zeros((1, 3))
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_particles_add_to(h, 1, r, V, one(5.0), one(0.5), one(0.2))
    assert ei.value.status == lbp.LBP_EINVAL
    lbp.lbp_particles_add_to(h, 2, r, V, one(5.0), one(0.5), one(0.2))
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_particles_add_to(h, len(BOXES), r, V, one(5.0), one(0.5), one(0.2))
    assert ei.value.status == lbp.LBP_EINVAL
    assert lbp.lbp_particles_count(h) == 1
    # a state update is checked against each particle's own box
    with pytest.raises(lbp.LbpError):
        lbp.lbp_particles_set_state(h, r=np.array([[131.0, 1.0, 1.0]]))
    lbp.lbp_particles_set_state(h, r=np.array([[129.5, 4.5, 3.5]]))
    lbp.lbp_destroy(h)


def test_per_particle_vacf_sums_and_trajectory():
    h = make_batch(lbp.LBP_F32, 1e-4, True)
    n = lbp.lbp_particles_count(h)
    K, T = 70, 150
    lbp.lbp_vacf_configure_ex(h, K, 1)
    traj = np.empty((T, n, 3))
    V = np.empty((n, 3))
    for t in range(T):
        lbp.lbp_step(h, 1)
        lbp.lbp_particles_read(h, v=V)
        traj[t] = V
    cs = np.empty((n, K + 1))
    cnt = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read_per_particle(h, cs, cnt)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_vacf_read(h, np.empty(K + 1), np.empty(K + 1, np.int64))
    assert ei.value.status == lbp.LBP_ESTATE
    lbp.lbp_destroy(h)
    assert np.array_equal(cnt, T - np.arange(K + 1))
    t32 = traj.astype(np.float32).astype(np.float64)
    ref = np.empty((n, K + 1))
    for k in range(K + 1):
        ref[:, k] = np.einsum("tic,tic->i", t32[k:], t32[:T - k])
    # FP32 products and block sums of at most 192 terms: relative 1e-5 of C_i(0)
    scale = ref[:, :1]
    assert np.all(np.abs(cs - ref) <= 1e-5 * scale + 1e-30)
    # the per-particle and the ensemble estimators agree
    h = make_batch(lbp.LBP_F32, 1e-4, True)
    lbp.lbp_vacf_configure(h, K)
    lbp.lbp_step(h, T)
    tot = np.empty(K + 1)
    cnt2 = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, tot, cnt2)
    lbp.lbp_destroy(h)
    assert np.array_equal(cnt2, n * cnt)
    assert np.max(np.abs(tot - cs.sum(axis=0))) <= 1e-5 * tot[0]


def make_box(prec, kT, shape=(20, 18, 16, 0.8)):
    nx, ny, nz, tau = shape
    f, ps = box_state(0, shape)
    h = lbp.lbp_create(nx, ny, nz, tau, precision=prec)
    lbp.lbp_set_populations(h, f)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=kT, seed=5)
    return h


SHAPE_BOXES = {"20x18x16": (20, 18, 16, 0.8), "24x10x9": (24, 10, 9, 0.7), "136x5x4": (136, 5, 4, 0.9),
               "22x6x5": (22, 6, 5, 0.8), "4x6x5": (4, 6, 5, 0.8)}


@pytest.mark.parametrize("prec", [lbp.LBP_F32, lbp.LBP_BF16, lbp.LBP_F16])
@pytest.mark.parametrize("where", ["20x18x16", "24x10x9", "136x5x4", "22x6x5", "4x6x5", "batch"])
def test_kernel_shapes_and_autotune_leave_results_unchanged(prec, where):
    """Every kernel shape -- one node per thread with 1, 2, 4 rows; two nodes
    per thread (2-byte storage, even nx); the bulk-copy staged kernel (nx a
    multiple of 16 bytes of storage); four nodes per thread (2-byte storage,
    nx a multiple of 4) -- and the autotuner's pick give bitwise the same run.
    The boxes cover ragged segments (136 = 128 + 8), periodic halos at both
    ends of a row, a row of one four-node group (nx = 4), nx = 22 (pairs but
    no groups of four), and the uneven batch (nx = 33 in one box: variant 0
    only)."""
    steps = 25
    batch = where == "batch"
    H = 4 if prec == lbp.LBP_F32 else 8
    nxs = [b[0] for b in BOXES] if batch else [SHAPE_BOXES[where][0]]
    ok = {0: True, 1: prec != lbp.LBP_F32 and all(n % 2 == 0 for n in nxs), 2: all(n % H == 0 for n in nxs),
          3: prec != lbp.LBP_F32 and all(n % 4 == 0 for n in nxs)}
    shapes = [(r, v) for v in (0, 1) if ok[v] for r in (1, 2, 4)] + ([(1, 2)] if ok[2] else []) + \
        [(r, 3) for r in (1, 2, 4) if ok[3]] + ["auto"]
    ref = None
    for shape in shapes:
        h = make_batch(prec, 1e-4, True) if batch else make_box(prec, 1e-4, SHAPE_BOXES[where])
        lbp.lbp_step(h, 3)
        if shape == "auto":
            rows, variant, ms = lbp.lbp_autotune(h, 5)
            valid = [m for m in ms if m > 0]
            assert len(valid) == 3 * ok[0] + 3 * ok[1] + ok[2] + 3 * ok[3]
            k = lbp.AUTOTUNE_SHAPES.index((variant, 1 if variant == 2 else rows))
            assert ms[k] == min(valid)
            want = (rows, variant)
        else:
            lbp.lbp_set_block_shape(h, *shape)
            want = shape
        d = lbp.lbp_diagnostics(h)
        assert (d["rows_per_block"], d["variant"]) == want
        assert lbp.lbp_get_step_index(h) == 3
        lbp.lbp_step(h, steps)
        lbp.lbp_check(h)
        got = read_batch(h)
        lbp.lbp_destroy(h)
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]), shape
            for k in range(4):
                assert np.array_equal(got[1][k], ref[1][k]), (shape, k)
    for v in (1, 2, 3):
        if not ok[v]:
            h = make_batch(prec, 0.0, True) if batch else make_box(prec, 0.0, SHAPE_BOXES[where])
            with pytest.raises(lbp.LbpError):
                lbp.lbp_set_block_shape(h, 1, v)
            lbp.lbp_destroy(h)


@pytest.mark.parametrize("prec", [lbp.LBP_F32, lbp.LBP_BF16, lbp.LBP_F16])
def test_default_kernel_shape(prec):
    """Before any lbp_autotune a handle runs the shape the autotuner picks at
    256^3: two rows of one node per thread for FP32, four nodes per thread for
    the 2-byte types where every nx is a multiple of 4 (else two rows of one)."""
    for box, quad in ((SHAPE_BOXES["20x18x16"], True), (SHAPE_BOXES["22x6x5"], False)):
        h = make_box(prec, 0.0, box)
        d = lbp.lbp_diagnostics(h)
        want = (1, 3) if prec != lbp.LBP_F32 and quad else (2, 0)
        assert (d["rows_per_block"], d["variant"]) == want, box
        lbp.lbp_destroy(h)
    h = make_batch(prec, 0.0, True)  # nx = 33 in one box: no four-node kernel
    d = lbp.lbp_diagnostics(h)
    assert (d["rows_per_block"], d["variant"]) == (2, 0)
    lbp.lbp_destroy(h)


def test_block_rows_validation():
    h = make_batch(lbp.LBP_F32, 0.0, True)
    with pytest.raises(lbp.LbpError):
        lbp.lbp_set_block_rows(h, 3)
    lbp.lbp_destroy(h)


def test_adjoint_of_a_batch_equals_its_boxes_alone():
    """Reverse-mode gradients of a batch (lbp_adjoint_record / _backward on the
    ensemble of uneven boxes, one of them without particles) equal, bit for
    bit, those of every box recorded and run back alone: dL/dtau per box, the
    particles' gamma, R, M, V0 and r0 gradients and dL/df0 on each box's
    nodes; the particle-free box gets exactly zero (the loss does not depend on
    it).  No noise, so that a particle's Philox counter (its index in the
    handle) plays no part."""
    steps, C = 30, 7
    h = make_batch(lbp.LBP_F32, 0.0, True)
    n = lbp.lbp_particles_count(h)
    rng = np.random.default_rng(3)
    gv = rng.normal(0.0, 1.0, (steps, n, 3))
    gr = rng.normal(0.0, 1.0, (steps, n, 3))
    vt = np.empty((steps, n, 3))
    lbp.lbp_adjoint_record(h, steps, C, v_traj=vt)

    def grads(nb, N):
        return {"tau": None, "gamma": np.zeros(nb), "radius": np.zeros(nb), "mass": np.zeros(nb),
                "v0": np.zeros((nb, 3)), "r0": np.zeros((nb, 3)), "f0": np.zeros((Q, N))}
    out = grads(n, h.N)
    out["tau"] = np.zeros(len(BOXES))
    lbp.lbp_adjoint_backward(h, steps, gv, gr, out)
    lbp.lbp_destroy(h)
    p0 = node0 = 0
    for b, box in enumerate(BOXES):
        nx, ny, nz, tau = box
        Nb = nx * ny * nz
        nb = NPART[b]
        fb = out["f0"][:, node0:node0 + Nb]
        if nb == 0:
            assert out["tau"][b] == 0.0 and not np.any(fb)
        else:
            f, ps = box_state(b, box)
            hb = lbp.lbp_create(nx, ny, nz, tau)
            lbp.lbp_set_populations(hb, f)
            lbp.lbp_particles_add(hb, ps.r, ps.V, ps.M, ps.gamma, ps.R)
            lbp.lbp_particles_set_params(hb, kT=0.0, seed=5)
            vb = np.empty((steps, nb, 3))
            lbp.lbp_adjoint_record(hb, steps, C, v_traj=vb)
            ob = grads(nb, Nb)
            ob["tau"] = np.zeros(1)
            lbp.lbp_adjoint_backward(hb, steps, np.ascontiguousarray(gv[:, p0:p0 + nb]),
                                     np.ascontiguousarray(gr[:, p0:p0 + nb]), ob)
            lbp.lbp_destroy(hb)
            assert np.array_equal(vb, vt[:, p0:p0 + nb]), b
            assert ob["tau"][0] == out["tau"][b], b
            for k in ("gamma", "radius", "mass", "v0", "r0"):
                assert np.array_equal(ob[k], out[k][p0:p0 + nb]), (b, k)
            assert np.array_equal(ob["f0"], fb), b
            assert ob["tau"][0] != 0.0
        p0 += nb
        node0 += Nb


def test_batch_boxes_against_the_oracle():
    """Three boxes of different sizes and relaxation times (tau = 0.6, 0.8, 1.0)
    with particles in one handle, each compared with the FP64 oracle of that
    box alone after 60 steps at the tolerances of the single-box coupled test
    (V and F_H to 1e-5 relative, r to 1e-6, populations to 1e-5 of the deviation
    scale).  kT = 0: a box's random force is keyed by the particle's index in
    the whole handle, which the oracle of one box does not share."""
    import oracle
    boxes = [(20, 18, 16, 0.6), (33, 7, 12, 0.8), (24, 10, 6, 1.0)]
    npart = [5, 3, 4]
    states = []
    for b, (nx, ny, nz, tau) in enumerate(boxes):
        f = wl.perturbed_populations(W, (nz, ny, nx), 0.02, 200 + b)
        ps = wl.uniform_particles(npart[b], (nz, ny, nx), 6.0, 0.5, 0.0, 0.0, 40 + b, 50 + b)
        ps.R = np.full(ps.n, wl.stokes_radius(0.5, tau))
        ps.V = np.random.default_rng(60 + b).normal(0.0, 0.01, (ps.n, 3))
        states.append((f, ps))
    h = lbp.lbp_create_batch(boxes)
    lbp.lbp_set_populations(h, np.concatenate([f.reshape(Q, -1) for f, _ in states], axis=1))
    for b, (_, ps) in enumerate(states):
        lbp.lbp_particles_add_to(h, b, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=0.0, seed=3)
    lbp.lbp_step(h, 60)
    lbp.lbp_check(h)
    N = sum(nx * ny * nz for nx, ny, nz, _ in boxes)
    fall = np.empty((Q, N))
    lbp.lbp_read_populations(h, fall)
    n = sum(npart)
    r, V, FH, FR = (np.empty((n, 3)) for _ in range(4))
    lbp.lbp_particles_read(h, r, V, FH, FR)
    lbp.lbp_destroy(h)
    off, p0 = 0, 0
    for b, (nx, ny, nz, tau) in enumerate(boxes):
        f, ps = states[b]
        o = oracle.Sim(nx, ny, nz, tau)
        o.set_fhat(f)
        o.add_particles(ps.r, ps.V, ps.M, ps.gamma, ps.R)
        o.set_params(kT=0.0, seed=3)
        o.step(60)
        ro, Vo, FHo, _ = o.particles()
        fo = o.fhat()
        o.close()
        sl = slice(p0, p0 + ps.n)
        assert np.max(np.abs(V[sl] - Vo)) <= 1e-5 * np.max(np.abs(Vo)), b
        assert np.max(np.abs(FH[sl] - FHo)) <= 1e-5 * np.max(np.abs(FHo)), b
        d = np.abs(r[sl] - ro)
        d = np.minimum(d, np.array([nx, ny, nz], float) - d)
        assert np.max(d) <= 1e-6, b
        fb = fall[:, off:off + nx * ny * nz].reshape(Q, nz, ny, nx)
        scale = np.max(np.abs(fo - W[:, None, None, None]))
        assert np.max(np.abs(fb - fo)) <= 1e-5 * scale + 1e-14, b
        off += nx * ny * nz
        p0 += ps.n


def test_largest_batch_of_256_boxes():
    """A batch of MAX_BATCH = 256 boxes of ragged sizes and four relaxation
    times in one handle (the replica table's search at both ends, the node and
    segment offsets of the last boxes): after 8 steps with graphs, boxes 0, 1,
    127, 128, 254, 255 and every box holding particles are bitwise equal to the
    same box run alone.  A 257th box is refused."""
    sizes = [(4, 4, 4), (8, 3, 5), (12, 6, 2), (20, 4, 3), (36, 2, 2), (132, 2, 1), (130, 3, 2), (9, 7, 3)]
    boxes = [(*sizes[b % len(sizes)], (0.6, 0.75, 0.9, 1.1)[b % 4]) for b in range(256)]
    npart = [3 if b % 37 == 0 or b == 255 else 0 for b in range(256)]

    def state(b):
        nx, ny, nz, tau = boxes[b]
        f = wl.perturbed_populations(W, (nz, ny, nx), 0.02, 500 + b)
        ps = wl.uniform_particles(npart[b], (nz, ny, nx), 6.0, 0.5, wl.stokes_radius(0.5, tau), 0.0,
                                  600 + b, 700 + b)
        return f, ps

    h = lbp.lbp_create_batch(boxes)
    assert lbp.lbp_replica_count(h) == 256
    lbp.lbp_set_populations(h, np.concatenate([state(b)[0].reshape(Q, -1) for b in range(256)], axis=1))
    for b in range(256):
        if npart[b]:
            _, ps = state(b)
            lbp.lbp_particles_add_to(h, b, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=0.0, seed=5)
    lbp.lbp_set_use_graphs(h, True)
    lbp.lbp_step(h, 8)
    lbp.lbp_check(h)
    f_all, parts = read_batch(h)
    lbp.lbp_destroy(h)
    node0 = np.cumsum([0] + [nx * ny * nz for nx, ny, nz, _ in boxes])
    p0 = np.cumsum([0] + npart)
    check = sorted({0, 1, 127, 128, 254, 255} | {b for b in range(256) if npart[b]})
    for b in check:
        nx, ny, nz, tau = boxes[b]
        f, ps = state(b)
        hb = lbp.lbp_create(nx, ny, nz, tau)
        lbp.lbp_set_populations(hb, f)
        if npart[b]:
            lbp.lbp_particles_add(hb, ps.r, ps.V, ps.M, ps.gamma, ps.R)
            lbp.lbp_particles_set_params(hb, kT=0.0, seed=5)
        lbp.lbp_step(hb, 8)
        lbp.lbp_check(hb)
        fb = np.empty((Q, nz * ny * nx))
        lbp.lbp_read_populations(hb, fb)
        assert np.array_equal(fb, f_all[:, node0[b]:node0[b + 1]]), b
        if npart[b]:
            pb = [np.empty((npart[b], 3)) for _ in range(4)]
            lbp.lbp_particles_read(hb, *pb)
            for a, c in zip(pb, parts):
                assert np.array_equal(a, c[p0[b]:p0[b + 1]]), b
        lbp.lbp_destroy(hb)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_create_batch(boxes + [(4, 4, 4, 0.8)])
    assert ei.value.status == lbp.LBP_EINVAL


@pytest.mark.parametrize("prec", [lbp.LBP_F32, lbp.LBP_BF16])
def test_fit_layouts_give_the_same_bits(prec):
    """The particle kernel fits Eq. 8 one lane per cell corner when there are
    few particles and one thread per particle when there are many; both sum
    the corners in the same tree order.  A small box inside a batch holding
    enough particles for the thread-per-particle layout evolves bit for bit
    like the same box alone, which takes the lane-per-corner layout."""
    steps = 20
    small = (16, 16, 16, 0.8)
    big = (128, 64, 64, 0.7)
    ps0 = wl.uniform_particles(20, (16, 16, 16), 6.0, 0.5, wl.stokes_radius(0.5, 0.8), 1e-4, 41, 42)
    ps1 = wl.uniform_particles(12000, (64, 64, 128), 6.0, 0.5, wl.stokes_radius(0.5, 0.7), 1e-4, 43, 44)
    f0 = wl.perturbed_populations(W, (16, 16, 16), 0.02, 45)
    f1 = wl.perturbed_populations(W, (64, 64, 128), 0.02, 46)

    hb = lbp.lbp_create_batch([small, big], precision=prec)
    lbp.lbp_set_populations(hb, np.concatenate([f0.reshape(Q, -1), f1.reshape(Q, -1)], axis=1))
    lbp.lbp_particles_add_to(hb, 0, ps0.r, ps0.V, ps0.M, ps0.gamma, ps0.R)
    lbp.lbp_particles_add_to(hb, 1, ps1.r, ps1.V, ps1.M, ps1.gamma, ps1.R)
    lbp.lbp_particles_set_params(hb, kT=1e-4, seed=9)
    assert not lbp.lbp_diagnostics(hb)["fit_per_corner"]
    lbp.lbp_step(hb, steps)
    lbp.lbp_check(hb)
    fb, pb = read_batch(hb)
    lbp.lbp_destroy(hb)

    hs = lbp.lbp_create(16, 16, 16, 0.8, precision=prec)
    lbp.lbp_set_populations(hs, f0)
    lbp.lbp_particles_add(hs, ps0.r, ps0.V, ps0.M, ps0.gamma, ps0.R)
    lbp.lbp_particles_set_params(hs, kT=1e-4, seed=9)
    assert lbp.lbp_diagnostics(hs)["fit_per_corner"]
    lbp.lbp_step(hs, steps)
    lbp.lbp_check(hs)
    fs, psl = read_batch(hs)
    lbp.lbp_destroy(hs)

    n = 16 ** 3
    assert np.array_equal(fb[:, :n], fs)
    for k in range(4):
        assert np.array_equal(pb[k][:20], psl[k]), k
    assert np.any(pb[2][:20] != 0.0)  # the fit ran (F_H non-zero)
