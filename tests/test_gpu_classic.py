"""Parity of the classic SZ ground truth (prediction from reconstructed
neighbours, Section "Prediction-Based Transformation") with the oracle's
point-by-point walk in storage order.

Codes, histogram, escapes, Huffman cost, stream bits and every
reconstructed value must match bit for bit: both sides take each decision
in float32 with the same operation order.  SSE: both sides sum the same
exactly computed float64 squares, the oracle in storage order and the GPU
in a fixed per-CTA order, so they differ by rounding order only: at most
the recursive-summation bound (N - 1) u relative (u = 2^-53) on the
oracle's side, taken here as max(1e-12, N 2^-52).  The GPU keeps the
largest error as a float32 (relative 2^-24); PSNR within 1e-6 relative.
"""
import math

import numpy as np
import pytest

import synth

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL_PSNR = 1e-6
REL_SSE = 1e-12  # floor of the summation-order bound, see rel_sse()
REL_MAXERR = 2.0 ** -24
EXACT = ["delta", "eb_sz", "sz_huff_gt", "sz_nsym_gt", "sz_nesc_gt", "sz_bits_gt", "br_sz_gt",
         "flags"]


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


def _fields():
    rng = np.random.default_rng(7)
    f = {}
    f["1d_ragged"] = (synth.grf_np((4097,), -2.0, 11) * 3).astype(np.float32)
    f["2d_ragged"] = (synth.grf_np((61, 58), -3.0, 12) * 50 + 7).astype(np.float32)
    # 2D tiles of 32 x 32: several tiles with ragged tails on both axes
    f["2d_tiles"] = (synth.grf_np((100, 300), -3.0, 21) * 4).astype(np.float32)
    f["2d_flat"] = (synth.grf_np((5, 700), -2.5, 22)).astype(np.float32)
    f["2d_tall"] = (synth.grf_np((300, 7), -2.5, 23)).astype(np.float32)
    f["3d_ragged"] = (synth.grf_np((17, 22, 19), -3.0, 13) * 2).astype(np.float32)
    f["3d_tiles"] = synth.config2_field(seed=14, shape=(24, 40, 44))
    f["3d_noise"] = rng.standard_normal((12, 16, 20)).astype(np.float32)
    f["3d_thin"] = (synth.grf_np((1, 40, 33), -3.0, 24)).astype(np.float32)
    # 3D tiles of one plane x 32 x 32: several in rows and columns, ragged
    f["3d_multi_tile"] = (synth.grf_np((3, 70, 260), -3.0, 25) * 9).astype(np.float32)
    fill = synth.grf_np((48, 64), -3.0, 15)
    f["2d_fill"] = synth.fill_region_np(fill, seed=16)
    return f


FIELDS = _fields()


def rel_sse(n):
    return max(REL_SSE, n * 2.0 ** -52)


def check(R, ctx, x, op, eb_sz):
    xd = torch.from_numpy(x).cuda()
    rec = torch.empty_like(xd)
    g = ctx.ground_truth_classic(xd, _gp(R, op), eb_sz, recon=rec)
    o = O.classic_sz(x, op, eb_sz, want_recon=True)
    for k in EXACT:
        assert g[k] == o[k], (k, g[k], o[k])
    assert _rel(g["psnr_sz_gt"], o["psnr_sz_gt"]) <= REL_PSNR
    assert _rel(g["sse_sz"], o["sse_sz"]) <= rel_sse(x.size), (g["sse_sz"], o["sse_sz"])
    assert _rel(g["maxerr_sz"], o["maxerr_sz"]) <= REL_MAXERR
    r = rec.cpu().numpy()
    if o["flags"] & R.RD_F_CONSTANT:
        np.testing.assert_array_equal(r, x)
    else:
        np.testing.assert_array_equal(r.view(np.uint32), o["recon"].view(np.uint32))
    # every reconstructed value within the bound
    assert np.all(np.abs(x.astype(np.float64) - r.astype(np.float64)) <= eb_sz)
    return g, o


@pytest.mark.parametrize("name", sorted(FIELDS))
@pytest.mark.parametrize("rel_eb,radius", [(1e-2, 32768), (1e-4, 32768), (1e-3, 8)])
def test_classic_matches_oracle(R, ctx, name, rel_eb, radius):
    x = FIELDS[name]
    vr = float(x.max()) - float(x.min())
    op = O.params(eb=1e-3, quant_radius=radius)
    g, o = check(R, ctx, x, op, rel_eb * vr)
    if radius == 8:
        assert o["sz_nesc_gt"] > 0  # the radius forces escapes


@pytest.mark.parametrize("shape", [(1,), (3,), (2, 3), (1, 1, 5), (5, 1, 1), (4, 4, 4), (33, 129),
                                   (2, 33, 129), (4, 1, 300), (3, 300, 1)])
def test_classic_tiny_and_edge_shapes(R, ctx, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape).astype(np.float32)
    op = O.params(eb=1e-3)
    check(R, ctx, x, op, 1e-2)


def test_classic_constant_field(R, ctx):
    x = np.full((9, 13), -2.5, np.float32)
    g, o = check(R, ctx, x, O.params(eb=1e-3), 1e-3)
    assert g["flags"] & R.RD_F_CONSTANT and math.isinf(g["psnr_sz_gt"])


def test_classic_subnormal_and_mixed_magnitudes(R, ctx):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((40, 50)).astype(np.float32)
    x[::3] *= np.float32(1e-38)
    x[1::7] *= np.float32(1e20)
    check(R, ctx, x, O.params(eb=1e-3), 1e-30)
    check(R, ctx, x, O.params(eb=1e-3), 1e12)


def test_classic_host_field_and_repeats(R, ctx):
    """A host field (staged), then repeats of the same call: the third is
    replayed from its CUDA graph; every result is the same, and the launch
    count is 6 + the wavefront launches per call (the finish step runs in
    the Huffman launch)."""
    x = FIELDS["2d_tiles"]
    op = O.params(eb=1e-3)
    gp = _gp(R, op)
    first = ctx.ground_truth_classic(x, gp, 0.01)
    xd = torch.from_numpy(x).cuda()
    waves = -(-100 // 32) + -(-300 // 32) - 1
    outs = []
    for _ in range(3):
        n0 = ctx.launch_count()
        outs.append(ctx.ground_truth_classic(xd, gp, 0.01))
        assert ctx.launch_count() - n0 == 6 + waves
    for o in outs:
        assert o == first


def test_classic_invalid_bound_and_budget(R):
    x = torch.from_numpy(FIELDS["3d_ragged"]).cuda()
    op = O.params(eb=1e-3)
    with R.Context(0) as c:
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(R.RdselError) as e:
                c.ground_truth_classic(x, _gp(R, op), bad)
            assert e.value.code == R.RD_ERR_INVALID_ARG
    # the reconstruction buffer counts against the context's budget
    big = torch.zeros((256, 256, 64), dtype=torch.float32, device="cuda")
    big[0, 0, 0] = 1.0
    with R.Context(0, hbm_budget=4 << 20) as c:
        c.ground_truth_classic(x, _gp(R, op), 1e-3)
        with pytest.raises(R.RdselError) as e:
            c.ground_truth_classic(big, _gp(R, op), 1e-3)
        assert e.value.code == R.RD_ERR_BUDGET


def test_classic_against_dual_quantization_truth(R, ctx):
    """The two SZ truths at the same bound: the same bin, both within the
    bound, and stream sizes of the same order (the prequantised codes stand
    in for the classic predictor's)."""
    x = synth.config2_field(seed=3, shape=(32, 48, 40))
    vr = float(x.max()) - float(x.min())
    op = O.params(eb=1e-4, r_sp=1.0)
    xd = torch.from_numpy(x).cuda()
    eb_sz = 1e-4 * vr
    gc = ctx.ground_truth_classic(xd, _gp(R, op), eb_sz)
    gd = ctx.ground_truth(xd, _gp(R, op), eb_sz)
    assert gc["delta"] == gd["delta"]
    assert gc["maxerr_sz"] <= eb_sz and gd["maxerr_sz"] <= eb_sz
    assert 0.5 <= gc["sz_bits_gt"] / gd["sz_bits_gt"] <= 2.0


@pytest.mark.parametrize("kind", ["hurricane_100x500x500", "atm_1800x3600_fill"])
def test_classic_full_size_fields(R, ctx, kind):
    """The workload sizes of the bench: every code decision and reconstructed
    value of the 25M-point 3D field and of a 6.5M-point 2D field with a
    1e-20 fill region, against the oracle's sequential walk."""
    if kind.startswith("hurricane"):
        x = synth.config2_field()
    else:
        g = synth.grf_np((1800, 3600), -3.0, 41)
        x = synth.fill_region_np(g, seed=42)
    vr = float(x.max()) - float(x.min())
    check(R, ctx, x, O.params(eb=1e-4), 1e-4 * vr)
