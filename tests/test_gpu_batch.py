"""Batched estimate (rd_select_batch) through the C ABI.

Each field's record must equal the per-field rd_select record on that field
alone, bit for bit (the same integer sums and the same fixed-order float64
steps), and through it the oracle's; the work split chosen by the autotuner
or forced, and CUDA-graph replay, must not change any result; a failing
field must fail alone."""
import numpy as np
import pytest

import synth

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL_PSNR = 1e-6
REL_ENTROPY = 1e-10
REL_SSE = 1e-6
EXACT_RESULT = ["vmin", "vmax", "vr", "eb_abs", "r_sp_eff", "minexp", "n_blocks",
                "n_sampled_blocks", "zfp_s2", "zfp_npoints", "zfp_ncoeff", "mse_sp", "br_zfp",
                "delta", "sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff",
                "selection", "flags"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_08901_gb300 import _build, rdsel

    _build.build()
    return rdsel


@pytest.fixture(scope="module")
def ctx(R):
    c = R.Context(0)
    yield c
    c.close()


def _rel(a, b):
    if a == b:
        return 0.0
    return abs(a - b) / max(abs(a), abs(b))


def _fields():
    f = []
    f.append((synth.grf_np((4097,), -2.0, 11) * 3).astype(np.float32))
    f.append(synth.config1_field())
    f.append((synth.grf_np((61, 58), -3.0, 12) * 50 + 7).astype(np.float32))
    f.append((synth.grf_np((17, 22, 19), -3.0, 13) * 2).astype(np.float32))
    f.append(synth.config2_field(seed=14, shape=(24, 40, 44)))
    f.append(np.full((33, 20), 3.0, dtype=np.float32))  # constant
    f.append(synth.fill_region_np(synth.grf_np((48, 64), -3.0, 15), seed=16))
    f.append(synth.config2_field(seed=17, shape=(50, 125, 130)))  # many work items
    f.append((synth.grf_np((600, 700), -2.5, 18) * 10).astype(np.float32))
    return f


FIELDS = _fields()
SETTINGS = [(1e-2, 1.0, 0, 0), (1e-4, 0.05, 1, 0), (1e-6, 0.2, 0, 1), (1e-3, 0.05, 0, 0),
            (1e-4, 0.1, 1, 1), (1e-4, 0.05, 0, 0), (1e-5, 0.25, 0, 0), (1e-4, 0.05, 0, 1),
            (1e-3, 0.01, 1, 0)]


def _params(R):
    return [R.params(eb=eb, r_sp=r, ec_mode=ec, sel_rule=sel) for eb, r, ec, sel in SETTINGS]


def _oparams(i):
    eb, r, ec, sel = SETTINGS[i]
    return O.params(eb=eb, r_sp=r, ec_mode=ec, sel_rule=sel)


@pytest.fixture(scope="module")
def dev_fields():
    return [torch.from_numpy(x).cuda() for x in FIELDS]


@pytest.fixture(scope="module")
def singles(R, ctx, dev_fields):
    ps = _params(R)
    return [ctx.select(x, p) for x, p in zip(dev_fields, ps)]


def test_batch_equals_per_field_select_and_oracle(R, ctx, dev_fields, singles):
    ctx.batch_set_config(None)
    res, tru, st = ctx.select_batch(dev_fields, _params(R))
    assert tru is None and st == [0] * len(FIELDS)
    for i, (g, s) in enumerate(zip(res, singles)):
        assert g == s, i
    # and the oracle, on the smaller fields
    for i, x in enumerate(FIELDS):
        if x.size > 2_000_000:
            continue
        o = O.select(x, _oparams(i))
        for k in EXACT_RESULT:
            assert res[i][k] == o[k], (i, k, res[i][k], o[k])
        for k in ("psnr_zfp", "psnr_sz"):
            assert _rel(res[i][k], o[k]) <= REL_PSNR, (i, k)
        for k in ("entropy", "br_sz"):
            assert _rel(res[i][k], o[k]) <= REL_ENTROPY, (i, k)


def test_autotuner_picks_a_candidate_split(R, ctx, dev_fields):
    ctx.batch_set_config(None)
    ctx.select_batch(dev_fields[:4], _params(R)[:4])
    cfg = ctx.batch_get_config()
    assert cfg["tuned"] == 1
    assert cfg["range_values"] in (1 << 16, 1 << 18, 1 << 20)
    assert cfg["zfp_blocks"] in (256, 1024, 4096)
    assert cfg["sz_blocks"] in (256, 1024, 4096)
    assert cfg["ctas"] == 0


@pytest.mark.parametrize("cfg", [
    {"range_values": 1 << 12, "zfp_blocks": 32, "sz_blocks": 8},
    {"range_values": 1 << 22, "zfp_blocks": 1 << 14, "sz_blocks": 1 << 14},
    {"range_values": 4100, "zfp_blocks": 77, "sz_blocks": 45, "ctas": 7},
    {"range_values": 1 << 16, "zfp_blocks": 1024, "sz_blocks": 1024, "ctas": 1},
])
def test_work_split_and_graph_replay_change_nothing(R, ctx, dev_fields, singles, cfg):
    ctx.batch_set_config(cfg)
    try:
        for rep in range(3):  # direct, captured, replayed
            res, _, st = ctx.select_batch(dev_fields, _params(R))
            assert st == [0] * len(FIELDS)
            for i, (g, s) in enumerate(zip(res, singles)):
                assert g == s, (rep, i)
        got = ctx.batch_get_config()
        assert got["tuned"] == 0 and got["range_values"] == (cfg["range_values"] + 3) // 4 * 4
    finally:
        ctx.batch_set_config(None)


def test_replay_launch_count(R, ctx, dev_fields):
    """reset, range, one sampled-blocks launch per dimensionality present,
    SZ histogram, code prep, final."""
    ps = _params(R)
    for _ in range(2):
        ctx.select_batch(dev_fields, ps)
    n0 = ctx.launch_count()
    ctx.select_batch(dev_fields, ps)
    dims = {x.dim() for x in dev_fields}
    assert ctx.launch_count() - n0 == 5 + len(dims)


def test_batch_truth_equals_evaluate(R, ctx, dev_fields):
    ps = _params(R)
    idx = [0, 1, 2, 3, 4, 5, 6]
    fs = [dev_fields[i] for i in idx]
    pl = [ps[i] for i in idx]
    res, tru, st = ctx.select_batch(fs, pl, truth=True)
    assert st == [0] * len(idx)
    for j, i in enumerate(idx):
        e, t = ctx.evaluate(dev_fields[i], ps[i])
        assert res[j] == e, i
        for k, v in t.items():
            if k in ("sse_sz", "sse_zfp"):
                assert _rel(tru[j][k], v) <= REL_SSE, (i, k)
            elif k in ("psnr_sz_gt", "psnr_zfp_gt"):
                assert _rel(tru[j][k], v) <= REL_PSNR, (i, k)
            else:
                assert tru[j][k] == v, (i, k, tru[j][k], v)


def test_failing_field_fails_alone(R, ctx, dev_fields, singles):
    bad = torch.from_numpy(FIELDS[2].copy()).cuda()
    bad[5, 7] = float("nan")
    fs = list(dev_fields[:4])
    fs[2] = bad
    ps = _params(R)[:4]
    with pytest.raises(R.RdselError) as ei:
        ctx.select_batch(fs, ps)
    assert ei.value.code == R.RD_ERR_NONFINITE
    res, _, st = ctx.select_batch(fs, ps, check=False)
    assert st == [0, 0, R.RD_ERR_NONFINITE, 0]
    assert res[2]["vr"] == 0.0 and res[2]["selection"] == 0
    for i in (0, 1, 3):
        assert res[i] == singles[i], i


def test_workspaces_reused_across_batches(R, ctx, dev_fields, singles):
    """The per-field tables are cleared by the passes that read them and
    fully only after a field stopped early: batches that reuse the same
    workspaces with other fields, after a failing field and after a
    constant one, give the per-field records."""
    ps = _params(R)
    bad = torch.from_numpy(FIELDS[2].copy()).cuda()
    bad[5, 7] = float("nan")
    const = torch.full((40, 50), 3.0, dtype=torch.float32, device="cuda")
    rounds = [
        ([dev_fields[0], dev_fields[1], bad, dev_fields[3]], [0, 1, None, 3]),
        ([dev_fields[0], dev_fields[1], dev_fields[2], dev_fields[3]], [0, 1, 2, 3]),
        ([dev_fields[4], const, dev_fields[6], dev_fields[7]], [4, None, 6, 7]),
        ([dev_fields[5], dev_fields[2], dev_fields[7], dev_fields[4]], [5, 2, 7, 4]),
        ([dev_fields[0], dev_fields[1], dev_fields[2], dev_fields[3]], [0, 1, 2, 3]),
    ]
    for fs, idx in rounds:
        pp = [ps[i] if i is not None else ps[0] for i in idx]
        res, _, st = ctx.select_batch(fs, pp, check=False)
        for k, i in enumerate(idx):
            if i is not None:
                assert st[k] == 0 and res[k] == singles[i], (idx, k)


def test_host_fields_are_rejected(R, ctx):
    with pytest.raises(R.RdselError) as ei:
        ctx.select_batch([FIELDS[1]], R.params())
    assert ei.value.code == R.RD_ERR_INVALID_ARG


def test_single_field_batch(R, ctx, dev_fields, singles):
    res, _, st = ctx.select_batch([dev_fields[4]], _params(R)[4])
    assert st == [0] and res[0] == singles[4]


def test_hot_code_batch_equals_per_field(R, ctx):
    """The batched residual histogram of a field whose codes are nearly all
    one value (a 16M-point sawtooth): the 16-bit window flushes before a
    counter wraps, and the record equals rd_select's and the oracle's."""
    n = 1 << 24
    x = (3 * (np.arange(n, dtype=np.int64) % 1000)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    p = R.params(eb=1e-3, r_sp=1.0)
    single = ctx.select(xd, p)
    res, _, st = ctx.select_batch([xd, xd], [p, p])
    assert st == [0, 0] and res[0] == single and res[1] == single
    o = O.select(x, O.params(eb=1e-3, r_sp=1.0))
    for k in EXACT_RESULT:
        assert single[k] == o[k], k
