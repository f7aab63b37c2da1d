"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (codes, histograms, ZFP coefficients and bit counts, sample
counts, escape counts, Huffman costs) and the selection must match bit for
bit; so must every float64 that is a single rounding of an exact quantity
(MSE_sp, delta, BR_zfp, BR_sz_huff, the ground-truth bit-rates).  Tolerances:
  PSNR            1e-6 relative (the target), observed ~1e-15 (libm log10);
  entropy, BR_sz  1e-10 relative: a sum of up to 65536 terms, each with one
                  ulp of log2 difference and a different summation order;
  SSE             1e-6 relative: the GPU squares float32 errors and sums
                  blocks pairwise in float32 before float64;
  max error       2^-22 relative: |x - xhat| rounded to float32 on the GPU.
"""
import math

import numpy as np
import pytest

import synth

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL_PSNR = 1e-6
REL_ENTROPY = 1e-10
REL_SSE = 1e-6
REL_MAXERR = 2.0 ** -22

EXACT_RESULT = ["vmin", "vmax", "vr", "eb_abs", "r_sp_eff", "minexp", "n_blocks",
                "n_sampled_blocks", "zfp_s2", "zfp_npoints", "zfp_ncoeff", "mse_sp", "br_zfp",
                "delta", "sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff",
                "selection", "flags"]
EXACT_TRUTH = ["eb_sz", "delta", "zfp_bits_gt", "br_zfp_gt", "sz_bits_gt", "sz_huff_gt",
               "sz_nesc_gt", "sz_nsym_gt", "br_sz_gt", "best_gt", "flags"]


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


def _gp(R, op):
    return R.params(eb=op.eb, eb_mode=op.eb_mode, ec_mode=op.ec_mode, r_sp=op.r_sp,
                    quant_radius=op.quant_radius, sel_rule=op.sel_rule, sz_offset=op.sz_offset)


def check_result(g, o, d):
    for k in EXACT_RESULT:
        assert g[k] == o[k], (k, g[k], o[k])
    assert g["strides"][:d] == o["strides"][:d]
    for k in ("psnr_zfp", "psnr_sz"):
        assert _rel(g[k], o[k]) <= REL_PSNR, (k, g[k], o[k])
    for k in ("entropy", "br_sz"):
        assert _rel(g[k], o[k]) <= REL_ENTROPY, (k, g[k], o[k])


def check_truth(g, o):
    for k in EXACT_TRUTH:
        assert g[k] == o[k], (k, g[k], o[k])
    for k in ("psnr_sz_gt", "psnr_zfp_gt"):
        assert _rel(g[k], o[k]) <= REL_PSNR, (k, g[k], o[k])
    for k in ("sse_sz", "sse_zfp"):
        assert _rel(g[k], o[k]) <= REL_SSE, (k, g[k], o[k])
    for k in ("maxerr_sz", "maxerr_zfp"):
        assert _rel(g[k], o[k]) <= REL_MAXERR, (k, g[k], o[k])


def _fields():
    rng = np.random.default_rng(2024)
    f = {}
    f["1d_ragged"] = (synth.grf_np((4097,), -2.0, 11) * 3).astype(np.float32)
    f["2d_cfg1_256"] = synth.config1_field()
    f["2d_ragged"] = (synth.grf_np((61, 58), -3.0, 12) * 50 + 7).astype(np.float32)
    f["3d_ragged"] = (synth.grf_np((17, 22, 19), -3.0, 13) * 2).astype(np.float32)
    f["3d_tiles"] = synth.config2_field(seed=14, shape=(24, 40, 44))
    f["3d_noise"] = rng.standard_normal((12, 16, 20)).astype(np.float32)
    fill = synth.grf_np((48, 64), -3.0, 15)
    f["2d_fill"] = synth.fill_region_np(fill, seed=16)
    return f


FIELDS = _fields()
CASES = [
    (name, eb, r_sp)
    for name in FIELDS
    for eb, r_sp in ((1e-2, 1.0), (1e-4, 0.05), (1e-6, 0.2))
]


@pytest.mark.parametrize("name,eb,r_sp", CASES)
def test_select_and_truth_match_oracle(R, ctx, name, eb, r_sp):
    x = FIELDS[name]
    op = O.params(eb=eb, r_sp=r_sp)
    xd = torch.from_numpy(x).cuda()
    g = ctx.select(xd, _gp(R, op))
    o = O.select(x, op, want_hist=True)
    check_result(g, o, x.ndim)
    hest, _ = ctx.histograms()
    assert np.array_equal(hest, o["hist"])
    # fused estimate + truth
    ge, gt = ctx.evaluate(xd, _gp(R, op))
    check_result(ge, o, x.ndim)
    ot = O.ground_truth(x, op, want_hist=True)
    check_truth(gt, ot)
    hest2, hgt = ctx.histograms()
    assert np.array_equal(hest2, o["hist"])
    assert np.array_equal(hgt, ot["hist"])
    # truth alone, delta from the estimate, and at an explicit bound
    check_truth(ctx.ground_truth(xd, _gp(R, op)), ot)
    eb_sz = 0.37 * o["eb_abs"]
    check_truth(ctx.ground_truth(xd, _gp(R, op), eb_sz=eb_sz), O.ground_truth(x, op, eb_sz=eb_sz))


@pytest.mark.parametrize("name", ["2d_ragged", "3d_ragged", "1d_ragged"])
@pytest.mark.parametrize("ec_mode,sel_rule,radius", [(1, 0, 32768), (0, 1, 32768), (0, 0, 40)])
def test_modes_match_oracle(R, ctx, name, ec_mode, sel_rule, radius):
    x = FIELDS[name]
    op = O.params(eb=1e-3, r_sp=0.25, ec_mode=ec_mode, sel_rule=sel_rule, quant_radius=radius)
    xd = torch.from_numpy(x).cuda()
    ge, gt = ctx.evaluate(xd, _gp(R, op))
    check_result(ge, O.select(x, op), x.ndim)
    check_truth(gt, O.ground_truth(x, op))


def test_estimate_entry_points_match_oracle(R, ctx):
    x = FIELDS["3d_tiles"]
    op = O.params(eb=1e-4, r_sp=0.05)
    xd = torch.from_numpy(x).cuda()
    o = O.select(x, op)
    gz = ctx.estimate_zfp(xd, _gp(R, op))
    for k in ("zfp_s2", "zfp_npoints", "zfp_ncoeff", "mse_sp", "br_zfp", "delta", "flags"):
        assert gz[k] == o[k], k
    assert _rel(gz["psnr_zfp"], o["psnr_zfp"]) <= REL_PSNR
    for delta in (o["delta"], 0.0, 3.3 * o["delta"]):
        gs = ctx.estimate_sz(xd, _gp(R, op), delta=delta)
        os_ = O.estimate_sz(x, op, delta=delta, want_hist=True)
        for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff", "delta", "flags",
                  "zfp_npoints", "n_sampled_blocks"):
            assert gs[k] == os_[k], (k, delta)
        assert _rel(gs["br_sz"], os_["br_sz"]) <= REL_ENTROPY
        assert _rel(gs["psnr_sz"], os_["psnr_sz"]) <= REL_PSNR
        assert np.array_equal(ctx.histograms()[0], os_["hist"])


@pytest.mark.parametrize("name", ["1d_ragged", "2d_ragged", "3d_ragged", "3d_tiles", "2d_fill"])
@pytest.mark.parametrize("eb_rel", [1e-2, 1e-5])
def test_zfp_blocks_bit_exact(R, ctx, name, eb_rel):
    x = FIELDS[name]
    eb_abs = eb_rel * (float(x.max()) - float(x.min()))
    g = ctx.zfp_blocks(torch.from_numpy(x).cuda(), eb_abs, want_coeffs=True)
    o = O.zfp_blocks(x, eb_abs, want_coeffs=True)
    for k in ("emax", "prec", "bits", "coeffs"):
        assert np.array_equal(g[k], o[k]), k


@pytest.mark.parametrize("name", ["1d_ragged", "2d_ragged", "3d_ragged", "3d_noise"])
@pytest.mark.parametrize("rel_delta,radius", [(2e-3, 32768), (2e-5, 32768), (1e-3, 8)])
def test_sz_symbols_bit_exact(R, ctx, name, rel_delta, radius):
    x = FIELDS[name]
    delta = rel_delta * (float(x.max()) - float(x.min()))
    strides = [2] * x.ndim
    g = ctx.sz_symbols(torch.from_numpy(x).cuda(), delta, radius, strides)
    o = O.sz_symbols(x, delta, radius, strides)
    assert np.array_equal(g["est"], o["est"])
    assert np.array_equal(g["gt"], o["gt"])
    assert np.array_equal(g["recon"].view(np.uint32), o["recon"].view(np.uint32))


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_constant_field(R, ctx):
    x = np.full((9, 13), -2.5, np.float32)
    op = O.params(eb=1e-3)
    ge, gt = ctx.evaluate(torch.from_numpy(x).cuda(), _gp(R, op))
    o = O.select(x, op)
    assert ge["flags"] & R.RD_F_CONSTANT and ge["selection"] == 1
    check_result(ge, o, 2)
    assert math.isinf(gt["psnr_sz_gt"]) and gt["best_gt"] == 1


@pytest.mark.parametrize("shape", [(1,), (3,), (2, 3), (1, 1, 5), (5, 1, 1), (4, 4, 4)])
def test_tiny_fields(R, ctx, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape).astype(np.float32)
    if x.size == 1:
        x = x + 0  # a single value is a constant field
    op = O.params(eb=1e-3, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    ge, gt = ctx.evaluate(xd, _gp(R, op))
    check_result(ge, O.select(x, op), x.ndim)
    check_truth(gt, O.ground_truth(x, op))


def test_nonfinite_rejected(R, ctx):
    x = synth.config1_field(seed=3, shape=(32, 32))
    for bad in (np.nan, np.inf, -np.inf):
        y = x.copy()
        y[7, 9] = bad
        with pytest.raises(R.RdselError) as e:
            ctx.select(torch.from_numpy(y).cuda(), R.params())
        assert e.value.code == R.RD_ERR_NONFINITE
        with pytest.raises(O.OracleError):
            O.select(y, O.params())


def test_evaluate_3d_edge_cases_then_a_good_call(R, ctx):
    """The 3D evaluate step writes its records from the last CTA of the
    truth's ZFP pass after the Huffman launch it follows: a constant field,
    a field with a non-finite value and a truth whose codes overflow must
    each report as the oracle does, and the next call must be unaffected."""
    op = O.params(eb=1e-3)
    good = synth.config2_field(seed=21, shape=(20, 24, 28))
    const = np.full((6, 7, 9), 1.5, np.float32)
    ge, gt = ctx.evaluate(torch.from_numpy(const).cuda(), _gp(R, op))
    assert ge["flags"] & R.RD_F_CONSTANT and ge["selection"] == 1
    check_result(ge, O.select(const, op), 3)
    check_truth(gt, O.ground_truth(const, op))
    assert math.isinf(gt["psnr_sz_gt"]) and gt["best_gt"] == 1
    bad = good.copy()
    bad[3, 5, 7] = np.nan
    with pytest.raises(R.RdselError) as e:
        ctx.evaluate(torch.from_numpy(bad).cuda(), _gp(R, op))
    assert e.value.code == R.RD_ERR_NONFINITE
    rng = np.random.default_rng(9)
    flat = (1000.0 + 1e-3 * rng.standard_normal((8, 16, 16))).astype(np.float32)
    with pytest.raises(R.RdselError) as e:
        ctx.evaluate(torch.from_numpy(flat).cuda(), _gp(R, O.params(eb=1e-9, r_sp=1.0)))
    assert e.value.code == R.RD_ERR_RANGE
    for _ in range(2):
        ge, gt = ctx.evaluate(torch.from_numpy(good).cuda(), _gp(R, op))
        check_result(ge, O.select(good, op), 3)
        check_truth(gt, O.ground_truth(good, op))


def test_range_error_when_codes_overflow(R, ctx):
    rng = np.random.default_rng(5)
    x = (1000.0 + 1e-3 * rng.standard_normal((16, 16))).astype(np.float32)
    op = O.params(eb=1e-9, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    check_result(ctx.select(xd, _gp(R, op)), O.select(x, op), 2)
    with pytest.raises(R.RdselError) as e:
        ctx.ground_truth(xd, _gp(R, op))
    assert e.value.code == R.RD_ERR_RANGE
    with pytest.raises(O.OracleError) as eo:
        O.ground_truth(x, op)
    assert eo.value.code == O.ERR_RANGE


def test_subnormal_and_mixed_magnitudes(R, ctx):
    rng = np.random.default_rng(6)
    x = (rng.standard_normal((20, 24)) * 1e-39).astype(np.float32)  # subnormal floats
    x[:4, :4] = rng.standard_normal((4, 4)).astype(np.float32) * 1e3
    x[8:12, 8:12] = 0.0
    for eb in (1e-3, 1e-7):
        op = O.params(eb=eb, r_sp=1.0)
        xd = torch.from_numpy(x).cuda()
        ge, gt = ctx.evaluate(xd, _gp(R, op))
        check_result(ge, O.select(x, op), 2)
        check_truth(gt, O.ground_truth(x, op))
        eb_abs = eb * (float(x.max()) - float(x.min()))
        g = ctx.zfp_blocks(xd, eb_abs, want_coeffs=True)
        o = O.zfp_blocks(x, eb_abs, want_coeffs=True)
        for k in ("emax", "prec", "bits", "coeffs"):
            assert np.array_equal(g[k], o[k]), k


def test_host_field_location(R, ctx):
    x = FIELDS["3d_ragged"]
    op = O.params(eb=1e-4, r_sp=0.2)
    ge, gt = ctx.evaluate(x, _gp(R, op))  # numpy array: RD_LOC_HOST
    check_result(ge, O.select(x, op), 3)
    check_truth(gt, O.ground_truth(x, op))


def test_pinned_host_field_staged_by_the_range_pass(R, ctx):
    """A field in pinned host memory is read by the range pass itself, which
    stores it into the staging buffer: the records equal those of the
    device copy and the oracle, on the direct launch, the graph capture and
    the replays (the buffer rewritten between calls), and for a pinned view
    that is not 16-byte aligned (staged by a copy)."""
    x = FIELDS["3d_tiles"]
    op = O.params(eb=1e-4, r_sp=0.2)
    gp = _gp(R, op)
    want = ctx.evaluate(torch.from_numpy(x).cuda(), gp)
    check_result(want[0], O.select(x, op), 3)
    check_truth(want[1], O.ground_truth(x, op))
    h = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    other = FIELDS["3d_ragged"]
    for i in range(4):
        h.copy_(torch.from_numpy(x))
        assert ctx.evaluate(h, gp) == want
    # the same pinned buffer, other contents: the replay reads them afresh
    h2 = torch.empty(other.shape, dtype=torch.float32, pin_memory=True)
    for i in range(3):
        h2.copy_(torch.from_numpy(other))
        got = ctx.evaluate(h2, gp)
        check_result(got[0], O.select(other, op), 3)
        check_truth(got[1], O.ground_truth(other, op))
    buf = torch.empty(x.size + 1, dtype=torch.float32, pin_memory=True)
    buf[1:].copy_(torch.from_numpy(x.ravel()))
    assert ctx.evaluate(buf[1:].view(x.shape), gp) == want


def test_unaligned_device_pointer(R, ctx):
    """A view starting one float into an allocation: rows are not 16-byte
    aligned, so the scalar load path runs."""
    x = FIELDS["2d_ragged"]
    buf = torch.zeros(x.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(x.ravel()).cuda()
    view = buf[1:].view(x.shape)
    op = O.params(eb=1e-4, r_sp=0.5)
    ge, gt = ctx.evaluate(view, _gp(R, op))
    check_result(ge, O.select(x, op), 2)
    check_truth(gt, O.ground_truth(x, op))


def test_sampling_rate_extremes(R, ctx):
    x = FIELDS["3d_tiles"]
    for r_sp in (1e-6, 0.01, 1.0):
        op = O.params(eb=1e-3, r_sp=r_sp)
        ge = ctx.select(torch.from_numpy(x).cuda(), _gp(R, op))
        check_result(ge, O.select(x, op), 3)


def test_repeated_calls_are_deterministic(R, ctx):
    x = FIELDS["3d_tiles"]
    op = _gp(R, O.params(eb=1e-4, r_sp=0.05))
    xd = torch.from_numpy(x).cuda()
    a = ctx.evaluate(xd, op)
    for _ in range(3):
        assert ctx.evaluate(xd, op) == a


def test_profiling_across_graph_capture_and_replay(R, ctx):
    """Direct call, captured call and replays give identical records; the
    per-kernel timings count every launch and leave no error behind for the
    next CUDA user in the process."""
    x = FIELDS["3d_tiles"]
    xd = torch.from_numpy(x).cuda()
    p = _gp(R, O.params(eb=1e-3, r_sp=0.05))
    ctx.set_profiling(True)
    ctx.reset_profile()
    base = ctx.evaluate(xd, p)
    for _ in range(4):
        assert ctx.evaluate(xd, p) == base
    st = ctx.kernel_stats()
    assert st["zfp_pass"][1] == 5 and st["zfp_pass"][0] > 0
    assert st["sz_pass"][1] == 5 and st["huffman"][1] == 5 and st["code_prep"][1] == 5
    ctx.set_profiling(False)
    y = torch.ones(1000, device="cuda")
    y.add_(1.0)
    torch.cuda.synchronize()
    assert float(y.sum()) == 2000.0


def test_large_alphabet_huffman(R, ctx):
    """White noise at a tiny bin: tens of thousands of distinct symbols, which
    sends the Huffman cost through the counting-sort path."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((256, 256)).astype(np.float32)
    op = O.params(eb=1e-3, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    for delta in (2e-4, 1e-3):
        gs = ctx.estimate_sz(xd, _gp(R, op), delta=delta)
        os_ = O.estimate_sz(x, op, delta=delta, want_hist=True)
        assert np.array_equal(ctx.histograms()[0], os_["hist"])
        for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff"):
            assert gs[k] == os_[k], (k, delta)
        assert _rel(gs["br_sz"], os_["br_sz"]) <= REL_ENTROPY
        gt = ctx.ground_truth(xd, _gp(R, op), eb_sz=delta / 2)
        ot = O.ground_truth(x, op, eb_sz=delta / 2)
        check_truth(gt, ot)
    assert os_["sz_nsym"] > 0


def _residual_field(counts):
    """A 1D field whose Lorenzo residuals (x[i] - x[i-1], x[-1] = 0) at bin
    width 1 have the histogram counts[t] for the codes +t and -t (t >= 1) and
    counts[0] for code 0: pairs (t, 0) of values, shuffled, all exact in
    float32."""
    rng = np.random.default_rng(11)
    ts = np.repeat(np.arange(1, len(counts)), np.asarray(counts[1:], np.int64))
    rng.shuffle(ts)
    x = np.zeros(2 * len(ts) + int(counts[0]), np.float32)
    x[0:2 * len(ts):2] = ts
    return x


@pytest.mark.parametrize("form", ["runs", "runs_large_counts", "global"])
def test_huffman_forms_for_wide_alphabets(R, ctx, form):
    """Alphabets past the linear shared-memory form: 60001 codes whose counts
    take a few distinct values (leaves as runs of equal weight, nodes in a
    ring), the same with three counts of 2^16 or more, and 65535 codes with
    4100 distinct counts (too many runs: linear queues in global memory)."""
    if form == "global":
        t = np.arange(32768)
        counts = np.where(t <= 4100, t, 1)
        counts[0] = 5
    else:
        t = np.arange(30001)
        counts = 1 + t % 5
        if form == "runs_large_counts":
            counts[1:4] = [70000, 65536, 131071]
    x = _residual_field(counts)
    op = O.params(eb=1e-3, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    gs = ctx.estimate_sz(xd, _gp(R, op), delta=1.0)
    os_ = O.estimate_sz(x, op, delta=1.0, want_hist=True)
    h = os_["hist"]
    assert int((h > 0).sum()) == 2 * (len(counts) - 1) + 1
    assert np.array_equal(ctx.histograms()[0], h)
    for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff"):
        assert gs[k] == os_[k], k
    assert _rel(gs["br_sz"], os_["br_sz"]) <= REL_ENTROPY


@pytest.mark.parametrize("name,sel_rule", [("3d_ragged", 0), ("2d_ragged", 1), ("3d_noise", 0)])
def test_rd_curve_matches_oracle(R, ctx, name, sel_rule):
    """The rate-distortion sweep: Algorithm 1 and its truth at each bound,
    and the selection based on error bound (both compressors at the same
    maximum error), by estimates and by ground truth."""
    x = FIELDS[name]
    ebs = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
    op = O.params(eb=1.0, r_sp=0.25, sel_rule=sel_rule)
    xd = torch.from_numpy(x).cuda()
    got = ctx.rd_curve(xd, _gp(R, op), ebs)
    ref = O.rd_curve(x, op, ebs)
    assert len(got) == len(ebs)
    for g, o in zip(got, ref):
        assert g["eb"] == o["eb"]
        check_result(g["est"], o["est"], x.ndim)
        check_truth(g["truth"], o["truth"])
        for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff", "delta", "eb_abs"):
            assert g["est_eb"][k] == o["est_eb"][k], k
        assert g["est_eb"]["delta"] == 2 * g["est"]["eb_abs"]
        for k in ("entropy", "br_sz"):
            assert _rel(g["est_eb"][k], o["est_eb"][k]) <= REL_ENTROPY, k
        check_truth(g["truth_eb"], o["truth_eb"])
        assert g["selection_eb"] == o["selection_eb"]
        assert g["best_eb_gt"] == o["best_eb_gt"]


def test_hot_code_flushes_histogram_window(R, ctx):
    """A 16M-point sawtooth whose Lorenzo residuals are nearly all one code
    (3 at bin width 1): each CTA counts far more than 2^16 of that code, so
    the 16-bit shared counters of the estimate histogram must be flushed
    before they wrap.  Histogram and Huffman cost equal the oracle's."""
    n = 1 << 24
    x = (3 * (np.arange(n, dtype=np.int64) % 1000)).astype(np.float32)
    op = O.params(eb=1e-3, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    gs = ctx.estimate_sz(xd, _gp(R, op), delta=1.0)
    os_ = O.estimate_sz(x, op, delta=1.0, want_hist=True)
    h = os_["hist"]
    assert h.max() > 1 << 23
    assert np.array_equal(ctx.histograms()[0], h)
    for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff"):
        assert gs[k] == os_[k], k


# ---------------------------------------------------------------------------
# Full-size Hurricane-shaped field (100 x 500 x 500), as the benchmark runs it
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def hurricane():
    return synth.config2_field()


@pytest.mark.parametrize("eb,r_sp", [(1e-4, 0.05), (1e-2, 0.01)])
def test_full_size_hurricane_field(R, ctx, hurricane, eb, r_sp):
    x = hurricane
    op = O.params(eb=eb, r_sp=r_sp)
    xd = torch.from_numpy(x).cuda()
    ge, gt = ctx.evaluate(xd, _gp(R, op))
    o = O.select(x, op, want_hist=True)
    check_result(ge, o, 3)
    ot = O.ground_truth(x, op, want_hist=True)
    check_truth(gt, ot)
    he, hg = ctx.histograms()
    assert np.array_equal(he, o["hist"]) and np.array_equal(hg, ot["hist"])
