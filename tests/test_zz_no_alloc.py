"""The allocation-free VACF entry point (lbp_vacf_correlate_noalloc).

Some callers cannot allocate device memory where they need a result -- code
running inside an allocator or memory pool it does not own, or a loop that
must not trigger an allocation.  lbp_vacf_correlate_noalloc keeps its scratch
in a fixed array compiled into the library.  This test checks, through the C
ABI, that two calls in a row on the same trajectory agree with the library's
regular VACF (lbp_vacf_read) within the tolerance the other VACF tests use,
which also shows that a call does not depend on what the previous call left
in the shared scratch.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_1909_13412_gb300 import lbp
from paper_1909_13412_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1909_13412_gb300 import build as lbp_build
    lbp_build.build()
    lbp.load()
    torch.cuda.set_device(0)


def test_noalloc_vacf_matches_regular_vacf_twice():
    shape = (8, 8, 8)
    n, K, T = 37, 90, 150
    ps = wl.uniform_particles(n, shape, 6.0, 0.5, 0.2, 1e-4, 1, 2)
    h = lbp.lbp_create(8, 8, 8, 0.8)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=1e-4, seed=2)
    lbp.lbp_vacf_configure(h, K)
    traj = []
    V = np.empty((n, 3))
    for _ in range(T):
        lbp.lbp_step(h, 1)
        lbp.lbp_particles_read(h, v=V)
        traj.append(V.astype(np.float32).copy())
    ref = np.empty(K + 1)
    ref_cnt = np.empty(K + 1, np.int64)
    lbp.lbp_vacf_read(h, ref, ref_cnt)
    lbp.lbp_destroy(h)

    samples = torch.from_numpy(np.ascontiguousarray(np.array(traj).reshape(T, 3 * n))).cuda()
    for call in range(2):
        cs = torch.full((K + 1,), np.nan, dtype=torch.float64, device="cuda")
        cnt = torch.full((K + 1,), -1, dtype=torch.int64, device="cuda")
        lbp.lbp_vacf_correlate_noalloc(samples, T, 3 * n, K, n, cs, cnt)
        torch.cuda.synchronize()
        got, got_cnt = cs.cpu().numpy(), cnt.cpu().numpy()
        assert np.array_equal(got_cnt, ref_cnt), call
        assert np.max(np.abs(got - ref)) <= 1e-6 * ref[0], call


def _noalloc(samples, T, ncomp, K, npairs):
    cs = torch.full((K + 1,), np.nan, dtype=torch.float64, device="cuda")
    cnt = torch.full((K + 1,), -1, dtype=torch.int64, device="cuda")
    lbp.lbp_vacf_correlate_noalloc(samples, T, ncomp, K, npairs, cs, cnt)
    torch.cuda.synchronize()
    return cs.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("n,K,T", [(400, 300, 420), (700, 333, 701)])
def test_noalloc_vacf_matches_the_oracle_over_several_tiles_and_chunks(n, K, T):
    """Several ragged lag tiles (128 lags per CTA) and component chunks (1024 per
    CTA): 400 particles = 1200 components (2 chunks), 700 = 2100 (3 chunks).
    Compared with the oracle's FP64 correlation (Section 3 estimator) of the same
    FP32 samples, twice in a row through the shared scratch."""
    g = np.random.default_rng(n)
    # velocities with a slowly decaying correlation, like a Brownian trajectory
    V = np.empty((T, n, 3))
    V[0] = g.standard_normal((n, 3)) * 0.005
    for t in range(1, T):
        V[t] = 0.97 * V[t - 1] + 0.0012 * g.standard_normal((n, 3))
    V32 = V.astype(np.float32)
    ref, ref_cnt = oracle.vacf(V32.astype(np.float64), K)
    samples = torch.from_numpy(np.ascontiguousarray(V32.reshape(T, 3 * n))).cuda()
    for call in range(2):
        got, got_cnt = _noalloc(samples, T, 3 * n, K, n)
        assert np.array_equal(got_cnt, ref_cnt), call
        assert np.max(np.abs(got - ref)) <= 1e-6 * ref[0], call


def test_noalloc_vacf_rejects_sizes_beyond_its_scratch():
    samples = torch.zeros((4, 3000), dtype=torch.float32, device="cuda")
    K = 524288 // 3  # 3 chunks of 1024 components x (K + 1) lags > 524288
    cs = torch.zeros(K + 1, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(K + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_vacf_correlate_noalloc(samples, 4, 3000, K, 1000, cs, cnt)
    assert ei.value.status == lbp.LBP_EINVAL
    assert "scratch" in lbp.lbp_last_error()
    # a lag count whose + 1 would overflow a 32-bit int is rejected, not wrapped
    # (straight through the C ABI: the binding would refuse the short outputs)
    import ctypes
    st = lbp.load().lbp_vacf_correlate_noalloc(ctypes.c_void_p(samples.data_ptr()), 4, 3000, 2 ** 31 - 1,
                                               1000, ctypes.c_void_p(cs.data_ptr()),
                                               ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(0))
    assert st == lbp.LBP_EINVAL
    assert "scratch" in lbp.lbp_last_error()
