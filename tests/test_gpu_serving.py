"""Serving loop (continuous batching of adaptive integrations) on the GPU."""
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
    return q, torch, q.GenvecTable.load()


def _drain(srv, ids, max_steps=200):
    for _ in range(max_steps):
        if all(srv.status(i)["state"] == srv.DONE for i in ids):
            return
        srv.step()
    raise AssertionError("requests did not complete")


def _feyn(q, seed):
    return q.Integrand.polynomial(W.feynman_regular(seed))


def test_result_alone_equals_result_in_the_mix(env):
    q, torch, tab = env
    srv = q.Server(tab, memory_budget=256 << 20, max_slots=16, m=16)
    a = srv.submit(_feyn(q, 1), epsrel=3e-2, maxeval=5_000_000, seed=7)
    _drain(srv, [a])
    alone = srv.status(a)
    srv.close()
    srv = q.Server(tab, memory_budget=256 << 20, max_slots=16, m=16)
    ids = [srv.submit(_feyn(q, 10 + i), epsrel=10 ** -(1 + i % 3), maxeval=2_000_000, seed=i)
           for i in range(3)]
    c, w = W.genz_params(4, 6, 3)
    ids.append(srv.submit(q.Integrand.genz(4, c, w), epsrel=1e-6, maxeval=20_000_000, seed=3))
    srv.step()                                  # others already running when a arrives
    a2 = srv.submit(_feyn(q, 1), epsrel=3e-2, maxeval=5_000_000, seed=7)
    ids += [srv.submit(_feyn(q, 20 + i), epsrel=1e-2, maxeval=1_000_000, seed=20 + i) for i in range(2)]
    _drain(srv, ids + [a2])
    mixed = srv.status(a2)
    srv.close()
    for k in ("integral", "error", "n", "iterations", "evaluations"):
        assert mixed[k] == alone[k], k


def test_server_matches_adaptive_integrate(env):
    q, torch, tab = env
    c, w = W.genz_params(4, 5, 2)
    f = q.Integrand.genz(4, c, w)
    ref = q.integrate(f, tab, 1021, 16, ("korobov", 3), seed=5,
                      opts=q.options(epsrel=1e-8, epsabs=0.0, maxeval=10 ** 10))
    srv = q.Server(tab, memory_budget=256 << 20, max_slots=4, m=16)
    rid = srv.submit(f, epsrel=1e-8, epsabs=0.0, minn=1021, maxeval=10 ** 10, seed=5)
    _drain(srv, [rid])
    got = srv.status(rid)
    srv.close()
    assert got["integral"] == ref["integral"] and got["error"] == ref["error"]
    assert got["n"] == ref["n"] and got["iterations"] == ref["iterations"]


def test_concurrent_requests_through_non_monotone_tile_counts(env):
    """Many concurrent requests of two families that run to their evaluation budget: the
    largest admissible lattice (n = 974,707, 2257 tiles at m = 32) has fewer tiles than the
    one they end on (n = 886,097, 2261 tiles), so a reservation sized by the largest
    lattice alone let one request's partials overwrite its neighbour in the pool.  Each
    result must equal qmc_integrate with the same arguments, bit for bit."""
    q, torch, tab = env
    m, maxeval = 32, 32 * 974_707 + 1000
    srv = q.Server(tab, memory_budget=1 << 30, max_slots=64, m=m, step_evaluations=0)
    fs = []
    for i in range(24):
        if i % 2 == 0:
            c, w = W.product_peak_params(4, 100 + i)
            fs.append(q.Integrand.genz(2, c, w))
        else:
            c, w = W.genz_params(4, 4, 100 + i)
            fs.append(q.Integrand.genz(4, c, w))
    ids = [srv.submit(f, epsrel=1e-12, epsabs=0.0, minn=1021, maxeval=maxeval, seed=i)
           for i, f in enumerate(fs)]
    _drain(srv, ids)
    got = [srv.status(i) for i in ids]
    srv.close()
    # the budget admits n = 974,707 but, after the first lattice, stops the escalation at
    # n = 886,097: the lattice with more tiles than the largest admissible one
    assert all(g["n"] == 886_097 for g in got)
    for i, f in enumerate(fs):
        ref = q.integrate(f, tab, 1021, m, ("korobov", 3), seed=i,
                          opts=q.options(epsrel=1e-12, epsabs=0.0, maxeval=maxeval))
        for k in ("integral", "error", "n", "iterations", "evaluations"):
            assert got[i][k] == ref[k], (i, k, got[i][k], ref[k])


def test_integrate_with_a_table_ending_below_a_larger_tile_count(env):
    """qmc_integrate's workspace covers every lattice the adaptive loop may visit: with the
    table cut at n = 974,707 (2257 tiles at m = 32) an adaptive run starting at n = 886,097
    (2261 tiles) must pass the lattice sums' workspace check and agree with the full
    table's run (one iteration each: the budget is exactly one lattice)."""
    q, torch, tab = env
    c, w = W.product_peak_params(4, 7)
    f = q.Integrand.genz(2, c, w)
    keep = [i for i, n in enumerate(tab.n) if n <= 974_707]
    cut = q.GenvecTable(np.asarray(tab.n)[keep], np.asarray(tab.z)[keep])
    opts = q.options(epsrel=1e-12, epsabs=0.0, maxeval=32 * 886_097)
    a = q.integrate(f, cut, 886_097, 32, ("korobov", 3), seed=3, opts=opts)
    b = q.integrate(f, tab, 886_097, 32, ("korobov", 3), seed=3, opts=opts)
    assert a["n"] == b["n"] == 886_097 and a["iterations"] == b["iterations"] == 1
    assert a["integral"] == b["integral"] and a["error"] == b["error"]


def test_completion_queue_reports_each_request_once(env):
    """qmc_server_completed lists every finished request exactly once, in completion
    order, and agrees with the per-request state."""
    q, torch, tab = env
    srv = q.Server(tab, memory_budget=256 << 20, max_slots=8, m=16)
    ids = []
    for i in range(12):
        c, w = W.genz_params(4, 3 + i % 3, 40 + i)
        ids.append(srv.submit(q.Integrand.genz(4, c, w), epsrel=10.0 ** -(3 + i % 4),
                              maxeval=4_000_000, seed=i))
    seen = []
    for _ in range(400):
        srv.step()
        for rid in srv.completed():
            assert srv.status(rid)["state"] == srv.DONE
            seen.append(rid)
        if len(seen) == len(ids):
            break
    assert sorted(seen) == sorted(ids) and len(set(seen)) == len(seen)
    assert srv.completed() == []
    # a request that no table size admits completes at admission, with its error status
    c, w = W.genz_params(4, 3, 99)
    bad = srv.submit(q.Integrand.genz(4, c, w), epsrel=1e-3, minn=10 ** 15, maxeval=10 ** 7, seed=1)
    srv.step()
    assert srv.completed() == [bad]
    with pytest.raises(q.QMCError) as e:   # status reports QMC_ERR_N for it
        srv.status(bad)
    assert e.value.code == -3
    srv.close()


def test_memory_budget_limits_concurrency(env):
    q, torch, tab = env
    # each request reserves the complex partials of its largest lattice (n = 108863: tiles x
    # 32 shifts x 4 doubles) plus a few KB of coefficients and shifts; the fixed buffers
    # take ~20 KB: a budget of 2.5 requests' partials fits two, not three
    tiles, _ = q.sums_tile_count(108863, 32)
    per_request = tiles * 32 * 4 * 8
    srv = q.Server(tab, memory_budget=int(2.5 * per_request) + 64 * 1024, max_slots=8, m=32)
    ids = [srv.submit(_feyn(q, 40 + i), epsrel=1e-2, maxeval=4_000_000, seed=i) for i in range(6)]
    most = 0
    for _ in range(300):
        srv.step()
        p, a, free = srv.counts()
        most = max(most, a)
        if all(srv.status(i)["state"] == srv.DONE for i in ids):
            break
    done = all(srv.status(i)["state"] == srv.DONE for i in ids)
    srv.close()
    assert done
    assert most == 2


def test_step_budget_runs_short_requests_first(env):
    """With a per-step evaluation budget a short request that arrives behind a long one
    completes first, and both results equal those of the unbudgeted server."""
    q, torch, tab = env
    c, w = W.genz_params(4, 5, 8)
    short = q.Integrand.genz(4, c, w)
    results = {}
    for budget in (0, 1 << 20):
        srv = q.Server(tab, memory_budget=256 << 20, max_slots=8, m=16, step_evaluations=budget)
        big = srv.submit(_feyn(q, 2), epsrel=1e-12, maxeval=60_000_000, seed=4)
        srv.step()
        small = srv.submit(short, epsrel=1e-4, maxeval=10_000_000, seed=5)
        done_at = {}
        for step in range(400):
            for rid in (big, small):
                if rid not in done_at and srv.status(rid)["state"] == srv.DONE:
                    done_at[rid] = step
            if len(done_at) == 2:
                break
            srv.step()
        assert len(done_at) == 2
        results[budget] = (srv.status(big), srv.status(small), done_at[small] < done_at[big])
        srv.close()
    for k in ("integral", "error", "n", "evaluations"):
        assert results[0][0][k] == results[1 << 20][0][k], k
        assert results[0][1][k] == results[1 << 20][1][k], k
    assert results[1 << 20][2]


def test_server_rejects_bad_arguments(env):
    q, torch, tab = env
    with pytest.raises(q.QMCError) as e:
        q.Server(tab, memory_budget=1 << 24, max_slots=4, m=1)
    assert e.value.code == -5
    srv = q.Server(tab, memory_budget=1 << 24, max_slots=4, m=8)
    with pytest.raises(q.QMCError):
        srv.submit(q.Integrand.trig(np.array([0.5]), np.array([1]), np.array([0.1])), epsrel=1e-3)
    srv.close()


def test_served_results_match_the_oracle_on_their_final_lattice(env):
    """Each served request ends on one lattice of the table (Sec. 3.3.1: results of the
    smaller lattices are discarded on escalation).  For real Genz and complex deformed
    requests served together, the final (Qbar, sigma) must equal the oracle's estimate on
    that lattice with the request's shifts (SplitMix64 seeded with its seed): Qbar within
    1e-12 of the mean |g| per component, sigma within max(1e-9 sigma, 2e-12 mean |g|)."""
    import oracle as O
    q, torch, tab = env
    m = 16
    reqs = []
    for i, (fam, d) in enumerate([(4, 5), (2, 4), (1, 6), (3, 3)]):
        c, w = W.genz_params(fam, d, 60 + i)
        reqs.append((q.Integrand.genz(fam, c, w), O.genz(fam, c, w), 10.0 ** -(4 + i % 3)))
    for i in range(3):
        fl = W.feynman_regular(70 + i, beta=0.6 if i % 2 == 0 else 0.95, lam=1.0)
        reqs.append((q.Integrand.polynomial(fl), O.feynman_complex(fl), 10.0 ** -(2 + i)))
    srv = q.Server(tab, memory_budget=256 << 20, max_slots=16, m=m)
    ids = [srv.submit(f, epsrel=eps, epsabs=0.0, minn=1021, maxeval=3_000_000, seed=80 + i)
           for i, (f, _, eps) in enumerate(reqs)]
    _drain(srv, ids, max_steps=400)
    got = [srv.status(i) for i in ids]
    srv.close()
    for i, ((f, of, eps), g) in enumerate(zip(reqs, got)):
        n = int(g["n"])
        assert n in tab and int(g["m"]) == m
        D = O.shifts(80 + i, m, f.dim)
        o = O.integrate(of, ("korobov", 3), n, tab.z_for(n)[:f.dim], D)
        A = o["A"].mean()
        assert abs(g["integral"].real - o["value_re"]) <= 1e-12 * A, (i, n)
        assert abs(g["error"].real - o["error_re"]) <= max(1e-9 * o["error_re"], 2e-12 * A), (i, n)
        if f.is_complex:
            assert abs(g["integral"].imag - o["value_im"]) <= 1e-12 * A, (i, n)
            assert abs(g["error"].imag - o["error_im"]) <= max(1e-9 * o["error_im"], 2e-12 * A), (i, n)
        else:
            assert g["integral"].imag == 0.0
