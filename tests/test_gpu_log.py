"""Parity of the log-scale quantisation estimate (rd_estimate_sz_log, Section
"Estimation Based on Static Quantization", log-scale case) with the oracle.

Bit for bit: the largest residual, the base b (both sides derive it on the
host from the same largest residual), the 65536-bin histogram, the number of
sampled points, the Huffman cost and the symbol count.  The float64 sums:
entropy within 1e-10 relative (terms added in another order), the bin-model
MSE within 1e-12 relative, PSNR within 1e-6 relative.
"""
import math

import numpy as np
import pytest

import synth
from test_gpu_parity import R, ctx, _gp  # noqa: F401

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return 0.0 if a == b else abs(a - b) / max(abs(a), abs(b))


def check_log(g, o):
    for k in ("vr", "eb_abs", "unit", "max_abs", "base", "ns", "huff_bits", "nsym", "flags"):
        assert g[k] == o[k], (k, g[k], o[k])
    for k in ("entropy", "br_log", "br_log_huff"):
        assert _rel(g[k], o[k]) <= 1e-10, (k, g[k], o[k])
    assert _rel(g["mse_log"], o["mse_log"]) <= 1e-12, (g["mse_log"], o["mse_log"])
    assert _rel(g["psnr_log"], o["psnr_log"]) <= 1e-6


def _fields():
    rng = np.random.default_rng(77)
    f = {}
    f["1d"] = (synth.grf_np((4099,), -2.0, 61) * 5).astype(np.float32)
    f["2d_ragged"] = (synth.grf_np((61, 58), -3.0, 62) * 50 + 7).astype(np.float32)
    f["3d_ragged"] = (synth.grf_np((17, 22, 19), -3.0, 63) * 2).astype(np.float32)
    f["3d_tiles"] = synth.config2_field(seed=64, shape=(24, 40, 44))
    f["3d_noise"] = rng.standard_normal((12, 16, 20)).astype(np.float32)
    f["2d_fill"] = synth.fill_region_np(synth.grf_np((48, 64), -3.0, 65), seed=66)
    return f


FIELDS = _fields()


@pytest.mark.parametrize("name", list(FIELDS))
@pytest.mark.parametrize("eb,r_sp,radius", [(1e-2, 1.0, 32768), (1e-4, 0.05, 32768),
                                            (1e-3, 0.2, 64)])
def test_log_estimate_matches_oracle(R, ctx, name, eb, r_sp, radius):
    x = FIELDS[name]
    op = O.params(eb=eb, r_sp=r_sp, quant_radius=radius)
    g = ctx.estimate_sz_log(torch.from_numpy(x).cuda(), _gp(R, op))
    o = O.estimate_sz_log(x, op, want_hist=True)
    check_log(g, o)
    hest, _ = ctx.histograms()
    assert np.array_equal(hest, o["hist"])


def test_log_estimate_special_cases(R, ctx):
    # constant field
    x = np.full((9, 10, 11), 2.5, np.float32)
    g = ctx.estimate_sz_log(torch.from_numpy(x).cuda(), R.params())
    assert g["flags"] & R.RD_F_CONSTANT and math.isinf(g["psnr_log"])
    # every residual inside the central bin: b = 1, one code
    w = np.zeros((40,), np.float32) + 2.0
    w[20:] = 3.0
    op = O.params(eb=4.0, eb_mode=O.EB_ABS, r_sp=1.0)
    g = ctx.estimate_sz_log(torch.from_numpy(w).cuda(), _gp(R, op))
    o = O.estimate_sz_log(w, op, want_hist=True)
    check_log(g, o)
    assert g["base"] == 1.0 and g["entropy"] == 0.0
    # a host field (staged) and a one-bin radius
    x = FIELDS["2d_ragged"]
    op = O.params(eb=1e-3, r_sp=0.5, quant_radius=1)
    check_log(ctx.estimate_sz_log(x, _gp(R, op)), O.estimate_sz_log(x, op))


def test_log_estimate_full_size_field(R, ctx):
    """The 100x500x500 Hurricane-shaped field at eb_rel 1e-4, r_sp 5%."""
    x = synth.config2_field()
    op = O.params(eb=1e-4, r_sp=0.05)
    g = ctx.estimate_sz_log(torch.from_numpy(x).cuda(), _gp(R, op))
    o = O.estimate_sz_log(x, op, want_hist=True)
    check_log(g, o)
    assert np.array_equal(ctx.histograms()[0], o["hist"])
