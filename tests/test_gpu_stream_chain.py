"""Back-to-back lattice sums on one stream.

The lattice-sum kernel, the tile reduction and the shift reduction are launched with
programmatic stream serialization, so each may be scheduled while its predecessor still
runs.  Every such kernel waits for its predecessor's completion before it touches memory;
this test checks the hazard that rule guards: many integrals issued back to back on one
stream share one workspace (each lattice-sum launch overwrites the partials the previous
integral's reduction reads), with no host synchronisation in between, and every result
must equal the same integral computed alone, bit for bit, in both orders of the queue."""
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


def _problems(env):
    q, torch, dev, tab = env
    out = []
    for i, (fam, d, n, tr) in enumerate([(4, 10, 108863, ("korobov", 3)), (1, 6, 4691, ("baker",)),
                                         (3, 8, 1072187, ("korobov", 1)), (2, 4, 1021, ("korobov", 2)),
                                         (4, 5, 108863, ("baker",)), (1, 10, 4691, ("korobov", 4))]):
        c, w = W.genz_params(fam, d, 300 + i)
        f = q.Integrand.genz(fam, c, w)
        D = torch.from_numpy(q.make_shifts(400 + i, 32, d).astype(np.int64)).to(dev)
        r = q.rule(n, tab.z_for(n)[:d], D, tr)
        out.append((f.device_struct(dev), r, n, D))
    return out


def _run(env, probs, order, sync_each):
    q, torch, dev, _ = env
    need = max(q.sums_workspace_bytes(r, False, 0, n) for _, r, n, _ in probs)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    sums = torch.zeros(len(probs), 4 * 32, dtype=torch.float64, device=dev)
    res = torch.zeros(len(probs), 4, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    for _ in range(3):
        for i in order:
            fd, r, n, _ = probs[i]
            q.sums(fd, r, 0, n, ws, sums[i], None, s)
            q.finalize(sums[i], 32, n, False, res[i], None, s)
            if sync_each:
                s.synchronize()
    torch.cuda.synchronize()
    return sums.cpu().numpy(), res.cpu().numpy()


def test_back_to_back_integrals_equal_isolated_ones(env):
    probs = _problems(env)
    ref_sums, ref_res = _run(env, probs, range(len(probs)), sync_each=True)
    for order in (range(len(probs)), reversed(range(len(probs)))):
        got_sums, got_res = _run(env, probs, list(order), sync_each=False)
        assert np.array_equal(got_sums, ref_sums)
        assert np.array_equal(got_res, ref_res)
    assert np.all(np.isfinite(ref_res[:, :2])) and np.all(ref_res[:, 1] > 0)
