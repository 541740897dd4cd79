"""The differentiable VACF estimator of the autograd module (CPU only).

adjoint.vacf computes every lag at once through the correlation theorem.  It
is held to the oracle's direct double sum over particles and time origins
(or_vacf, the estimator of Section 3 written out) and its gradient to
autograd through the same direct definition, lag by lag.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from paper_1909_13412_gb300 import adjoint  # noqa: E402


@pytest.mark.parametrize("T,n,K", [(1, 3, 0), (7, 1, 6), (50, 4, 17), (129, 5, 128), (300, 2, 40)])
def test_vacf_equals_the_direct_sum(T, n, K):
    V = np.random.default_rng(T + n).normal(0.0, 0.01, (T, n, 3))
    got = adjoint.vacf(torch.tensor(V), K).numpy()
    cs, cnt = oracle.vacf(V, K)
    want = cs / cnt
    assert np.allclose(got, want, rtol=0, atol=1e-13 * np.abs(want[0]))


def test_vacf_gradient_equals_the_direct_definition():
    g = np.random.default_rng(4)
    T, n, K = 90, 3, 31
    V = g.normal(0.0, 0.01, (T, n, 3))
    w = torch.tensor(g.normal(0.0, 1.0, K + 1))
    a = torch.tensor(V, requires_grad=True)
    (adjoint.vacf(a, K) * w).sum().backward()
    b = torch.tensor(V, requires_grad=True)
    direct = torch.stack([(b[k:] * b[:T - k]).sum(-1).mean() for k in range(K + 1)])
    (direct * w).sum().backward()
    assert torch.allclose(a.grad, b.grad, rtol=0, atol=1e-12 * b.grad.abs().max().item())


def test_vacf_refuses_lags_beyond_the_trajectory():
    V = torch.zeros((5, 2, 3), dtype=torch.float64)
    with pytest.raises(ValueError):
        adjoint.vacf(V, 5)
    with pytest.raises(ValueError):
        adjoint.vacf(V, -1)
