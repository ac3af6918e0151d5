"""qmc_sums_noalloc: the lattice sums for callers that cannot allocate device memory (code
under CUDA-graph capture, deployments that fix all device memory up front).  It must give
the same per-shift sums as qmc_sums with a caller workspace, call after call, although
every call reuses the library's one fixed device scratch array.

Collected last on purpose (file name), so a run that stops at the first failure has run
every other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest

import workloads as W

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
    return q, torch, torch.device("cuda:0"), q.GenvecTable.load()


def _problem(env, fam, d, n, m, seed, transform):
    q, torch, dev, tab = env
    if fam == "feynman":
        f = q.Integrand.polynomial(W.feynman_regular(seed, d=d))
    else:
        c, w = W.genz_params(fam, d, seed)
        f = q.Integrand.genz(fam, c, w)
    D = q.make_shifts(seed, m, d)
    Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
    r = q.rule(n, tab.z_for(n)[:d], Dd, transform)
    return f, f.device_struct(dev), r, Dd


def _with_workspace(env, f, fd, r, n):
    q, torch, dev, _ = env
    ws = torch.empty(q.sums_workspace_bytes(r, f.is_complex, 0, n), dtype=torch.uint8, device=dev)
    out = torch.zeros(4 * r.m, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    q.sums(fd, r, 0, n, ws, out, cnt)
    torch.cuda.synchronize()
    return out.cpu().numpy(), cnt.cpu().numpy()


def _without_workspace(env, fd, r, n):
    q, torch, dev, _ = env
    out = torch.zeros(4 * r.m, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    q.sums_noalloc(fd, r, 0, n, out, cnt)
    torch.cuda.synchronize()
    return out.cpu().numpy(), cnt.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(env):
    # a larger problem, then smaller ones of other families (the complex one with twice
    # the partials per tile): a call must not see the previous call's partials left in the
    # shared scratch.  Both entry points run the same kernels on the same tiling, so the
    # double-double sums (hi and lo words, real and imaginary parts) must agree bit for bit.
    cases = [(4, 10, 1072187, 32, 11, ("korobov", 3)),
             (1, 6, 108863, 16, 12, ("baker",)),
             ("feynman", 5, 108863, 32, 14, ("korobov", 3)),
             (3, 8, 4691, 10, 13, ("korobov", 2))]
    for fam, d, n, m, seed, tr in cases:
        f, fd, r, _keep = _problem(env, fam, d, n, m, seed, tr)
        ref, ref_cnt = _with_workspace(env, f, fd, r, n)
        got, got_cnt = _without_workspace(env, fd, r, n)
        k = (4 if f.is_complex else 2) * m
        assert np.array_equal(got[:k], ref[:k]), (fam, d, n)
        S_ref = ref[0:2 * m:2] + ref[1:2 * m:2]
        assert np.all(np.isfinite(S_ref)) and np.any(S_ref != 0.0)
        assert np.array_equal(got_cnt, ref_cnt)


def test_noalloc_rejects_problems_beyond_the_fixed_scratch(env):
    q, torch, dev, tab = env
    n, d, m = 10560653, 3, 1024
    _f, fd, r, _keep = _problem(env, 4, d, n, m, 21, ("baker",))
    assert q.sums_workspace_bytes(r, False, 0, n) > q._capi.QMC_NOALLOC_SCRATCH_BYTES
    out = torch.zeros(4 * m, dtype=torch.float64, device=dev)
    with pytest.raises(q.QMCError) as e:
        q.sums_noalloc(fd, r, 0, n, out)
    assert e.value.code == -10
    # nothing was written
    torch.cuda.synchronize()
    assert not out.any().item()
