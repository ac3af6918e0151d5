"""Fast CBC on the GPU (qmc_cbc_korobov) against the oracle's CBC constructions and the
shipped table (App. A.3 generating vectors).

e^2 = -1 + (1/n) sum_k prod_j (beta + gamma omega) is 1 minus a mean of n terms near 1, so
both sides carry absolute rounding errors of a few (log2 n) x 1.1e-16 (plus the FFT's
relative 1e-15 log2 n on the candidate sums): compared with rtol 1e-10 and atol 1e-13."""
import numpy as np
import pytest

from oracle import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1811_11720_gb300 as q
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1811_11720_gb300 import build
    build.build()
    q.lib()
    return q, q.GenvecTable.load(extension=False)


@pytest.mark.parametrize("n,s", [(7, 2), (11, 2), (101, 6), (211, 5), (1021, 10)])
def test_matches_brute_force_cbc(env, n, s):
    q, _ = env
    z, e2 = q.cbc_korobov(n, s)
    zo, eo = L.cbc_naive(n, s)
    assert [int(v) for v in z] == [int(v) for v in zo]
    assert np.allclose(e2, eo, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("n", [1021, 4691, 19583, 108863, 1072187])
def test_matches_table_and_error_definition(env, n):
    """Same vector as the CPU fast CBC that wrote the table; e^2 of the full vector equals
    the definition summed over all n points."""
    q, tab = env
    z, e2 = q.cbc_korobov(n, 10)
    assert [int(v) for v in z] == [int(v) for v in tab.z_for(n)]
    exact = L.worst_case_error_sq(n, [int(v) for v in z], s_weights=10)
    assert abs(e2[-1] - exact) <= 1e-10 * abs(exact) + 1e-13


def test_gamma_beta_arguments(env):
    q, _ = env
    n, s = 1021, 4
    z, e2 = q.cbc_korobov(n, s, gamma=0.5, beta=2.0)
    zo, eo = L.cbc_naive(n, s, beta=2.0, gamma=0.5)
    assert [int(v) for v in z] == [int(v) for v in zo]
    assert np.allclose(e2, eo, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("n,s", [(1, 2), (4, 2), (1023, 3), (1021, 0)])
def test_rejects_bad_arguments(env, n, s):
    q, _ = env
    with pytest.raises(q.QMCError) as e:
        q.cbc_korobov(n, s)
    assert e.value.code == -1
