"""The serving loop (rd_server_*) through the C ABI: requests served
concurrently, with resident fields admitted and evicted under an HBM
budget, give each the same record as rd_select on the field alone and as
the oracle (integers and singly rounded doubles exact, PSNR within 1e-6,
entropy within 1e-10 relative); errors stay with their request; the
counters and latency percentiles add up."""
import numpy as np
import pytest

import synth
from test_gpu_parity import check_result

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_08901_gb300 import _build, rdsel

    _build.build()
    return rdsel


def _population():
    f = []
    f.append(synth.config1_field())
    f.append((synth.grf_np((61, 58), -3.0, 12) * 50 + 7).astype(np.float32))
    f.append((synth.grf_np((17, 22, 19), -3.0, 13) * 2).astype(np.float32))
    f.append(synth.config2_field(seed=14, shape=(24, 40, 44)))
    f.append((synth.grf_np((4097,), -2.0, 11) * 3).astype(np.float32))
    f.append((synth.grf_np((300, 257), -2.5, 21)).astype(np.float32))
    f.append(synth.config2_field(seed=22, shape=(40, 64, 60)))
    f.append((synth.grf_np((33, 31, 29), -3.5, 23) * 1e3).astype(np.float32))
    return f


POP = _population()
SETTINGS = [(1e-2, 1.0), (1e-4, 0.05), (1e-3, 0.2), (1e-5, 0.05)]


def test_mixed_requests_match_alone(R):
    rng = np.random.default_rng(7)
    prms = [R.params(eb=eb, r_sp=r) for eb, r in SETTINGS]
    dev = [torch.from_numpy(x).cuda() for x in POP]
    with R.Context(0) as ctx:
        alone = {(i, j): ctx.select(dev[i], prms[j]) for i in range(len(POP)) for j in range(len(prms))}
    # a budget that holds about a third of the population, so that fields
    # are evicted and loaded again
    budget = max(sum(x.nbytes for x in POP) // 3, max(x.nbytes for x in POP))
    want = {}
    with R.Server(0, slots=4, window=6, hbm_budget=budget) as srv:
        for t in range(96):
            i = int(rng.integers(len(POP)))
            j = int(rng.integers(len(prms)))
            kind = t % 6
            if kind == 5:
                rid = srv.submit(dev[i], prms[j], key=0, tag=t)          # device field
            elif kind == 4:
                rid = srv.submit(POP[i], prms[j], key=0, tag=t)          # transient host copy
            else:
                rid = srv.submit(POP[i], prms[j], key=100 + i, tag=t)    # resident host copy
            want[rid] = (i, j)
        got = []
        while len(got) < len(want):
            got += srv.poll(64, wait_ms=2000)
        st = srv.stats()
    assert len(got) == len(want)
    oracle = {}
    for c in got:
        assert c["status"] == 0, c
        i, j = want[c["request_id"]]
        assert c["result"] == alone[(i, j)], (i, j)
        if (i, j) not in oracle:
            eb, r_sp = SETTINGS[j]
            oracle[(i, j)] = O.select(POP[i], O.params(eb=eb, r_sp=r_sp))
        check_result(c["result"], oracle[(i, j)], POP[i].ndim)
        assert c["latency_ms"] >= c["service_ms"] >= 0.0 and c["queue_ms"] >= 0.0
    assert st["submitted"] == st["completed"] == len(want)
    assert st["evictions"] > 0 and st["resident_hits"] > 0
    assert st["resident_bytes"] <= budget
    assert 0.0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_failing_request_fails_alone(R):
    bad = POP[1].copy()
    bad[3, 4] = np.nan
    p = R.params(eb=1e-4)
    with R.Server(0, slots=2, window=4) as srv:
        a = srv.submit(POP[0], p, key=1)
        b = srv.submit(bad, p, key=2)
        c = srv.submit(POP[2], p, key=3)
        got = []
        while len(got) < 3:
            got += srv.poll(8, wait_ms=2000)
    st = {g["request_id"]: g["status"] for g in got}
    assert st[a] == 0 and st[c] == 0 and st[b] == R.RD_ERR_NONFINITE


def test_field_over_budget_is_rejected(R):
    with R.Server(0, slots=1, window=1, hbm_budget=1024) as srv:
        with pytest.raises(R.RdselError) as ei:
            srv.submit(POP[0], R.params(), key=1)
        assert ei.value.code == R.RD_ERR_BUDGET
        assert srv.stats()["rejected"] == 1
