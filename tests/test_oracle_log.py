"""Pins of the oracle's log-scale quantisation estimate (Section "Estimation
Based on Static Quantization", the log-scale case), against exact rational
arithmetic, closed forms and the paper's own observations.

The reading (stated in the oracle): unit u = eb_abs, base b the smallest
double >= 1 with u * b^n above max |r|, edges A[k] = u * pow(b, k), code 0
for |r| < A[1] and sign(r) * #{k <= n-1 : A[k] <= |r|} otherwise, bin widths
2 A[1] and A[k+1] - A[k].
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth

O = pytest.importorskip("oracle")


def _ramp(codes):
    """1D field whose Lorenzo residuals are exactly `codes` (integers)."""
    x = np.cumsum(np.asarray(codes, dtype=np.int64))
    assert np.abs(x).max() < 2 ** 24
    return x.astype(np.float32)


def _pow_frac(b: float, k: int) -> Fraction:
    return Fraction(b) ** k


@pytest.mark.parametrize("n", [8, 64, 300])
def test_base_is_the_smallest_that_covers_the_largest_residual(n):
    """u b^n exceeds max|r| and u b'^n does not for the double b' below b,
    in exact arithmetic up to the two roundings of the edge."""
    rng = np.random.default_rng(n)
    codes = rng.integers(-5000, 5000, 4000)
    x = _ramp(codes)
    r = O.estimate_sz_log(x, O.params(eb=1.0, eb_mode=O.EB_ABS, r_sp=1.0, quant_radius=n),
                          want_edges=True)
    u, b, M = Fraction(r["unit"]), r["base"], Fraction(r["max_abs"])
    assert M == max(abs(int(c)) for c in codes)
    tol = Fraction(1, 2 ** 50)
    assert u * _pow_frac(b, n) > M * (1 - tol)
    bprev = math.nextafter(b, 0.0)
    assert b == 1.0 or u * _pow_frac(bprev, n) < M * (1 + tol)
    e = r["edges"]
    assert len(e) == n and np.all(np.diff(e) >= 0) and e[-1] > r["max_abs"]


@pytest.mark.parametrize("n", [16, 200])
def test_every_residual_lies_in_its_bin(n):
    """The histogram equals a classification of the known residuals against
    the exact edges u b^k (rationals), except for residuals within rounding
    of an edge; the bins are symmetric and cover every residual."""
    rng = np.random.default_rng(100 + n)
    codes = np.rint(rng.standard_normal(6000) * 300).astype(np.int64)
    x = _ramp(codes)
    p = O.params(eb=0.37, eb_mode=O.EB_ABS, r_sp=1.0, quant_radius=n)
    r = O.estimate_sz_log(x, p, want_hist=True, want_edges=True)
    u, b = Fraction(r["unit"]), r["base"]
    exact = [u * _pow_frac(b, k) for k in range(n + 1)]
    want = np.zeros(65536, np.int64)
    near = 0
    for c in codes:
        a = Fraction(abs(int(c)))
        k = 0
        for j in range(1, n):
            if exact[j] <= a:
                k = j
        if any(abs(a - exact[j]) <= a * Fraction(1, 2 ** 48) for j in range(1, n)):
            near += 1
        want[32768 + (k if c >= 0 else -k)] += 1
    got = r["hist"].astype(np.int64)
    assert int(got.sum()) == len(codes) and got[0] == 0
    assert np.abs(got - want).sum() <= 2 * near
    assert r["ns"] == len(codes)


def test_equal_counts_over_every_bin_give_log2_of_the_bin_count():
    """The equal-probability special case: residuals placed one per bin of
    each sign (2n - 1 bins), each repeated equally: entropy = log2(2n - 1)
    and BR_log = entropy + 0.5."""
    n = 8
    M = 150
    base = O.estimate_sz_log(_ramp([M, -M, 0, 0]),
                             O.params(eb=1.0, eb_mode=O.EB_ABS, r_sp=1.0, quant_radius=n),
                             want_edges=True)
    A = [base["unit"]] + list(base["edges"])  # A[0] = u
    picks = [0]
    for k in range(1, n):
        lo, hi = A[k], A[k + 1]
        v = M if k == n - 1 else int(math.ceil(math.sqrt(lo * hi)))
        assert lo <= v < hi, (k, lo, v, hi)
        picks += [v, -v]
    assert len(picks) == 2 * n - 1
    codes = np.tile(np.array(picks), 64)
    r = O.estimate_sz_log(_ramp(codes), O.params(eb=1.0, eb_mode=O.EB_ABS, r_sp=1.0,
                                                 quant_radius=n), want_hist=True)
    assert r["base"] == base["base"]
    h = r["hist"]
    assert np.count_nonzero(h) == 2 * n - 1 and np.all(h[h > 0] == 64)
    assert abs(r["entropy"] - math.log2(2 * n - 1)) <= 1e-14
    assert r["br_log"] == r["entropy"] + 0.5


def test_mse_and_psnr_follow_the_bin_model():
    """Eq. (mse-pdf) with the histogram as the PDF: MSE = sum h delta^2 /
    (12 N), summed exactly here; PSNR by Eq. (psnr-pdf)."""
    x = synth.config2_field(seed=41, shape=(12, 20, 24))
    p = O.params(eb=1e-3, r_sp=0.25, quant_radius=512)
    r = O.estimate_sz_log(x, p, want_hist=True, want_edges=True)
    A = [r["unit"]] + list(r["edges"])
    h = r["hist"]
    tot = Fraction(0)
    for s in np.nonzero(h)[0]:
        k = abs(int(s) - 32768)
        w = Fraction(2 * A[1]) if k == 0 else Fraction(A[k + 1]) - Fraction(A[k])
        tot += int(h[s]) * w * w
    mse = tot / (12 * int(h.sum()))
    assert abs(Fraction(r["mse_log"]) - mse) <= mse * Fraction(1, 10 ** 13)
    psnr = 20 * math.log10(r["vr"]) - 10 * math.log10(float(mse))
    assert abs(r["psnr_log"] - psnr) <= 1e-9 * psnr


@pytest.mark.parametrize("seed,eb", [(51, 1e-2), (52, 1e-3), (53, 1e-4)])
def test_log_scale_trades_rate_for_psnr_as_the_paper_says(seed, eb):
    """The paper: log-scale quantisation usually has a higher PSNR but a
    lower compression ratio than linear quantisation (finer bins where the
    residuals crowd, a flatter histogram).  Same residuals, same unit."""
    x = synth.config2_field(seed=seed, shape=(16, 32, 36))
    p = O.params(eb=eb, r_sp=1.0)
    lg = O.estimate_sz_log(x, p)
    li = O.estimate_sz(x, p)
    assert lg["psnr_log"] > li["psnr_sz"]
    assert lg["br_log"] > li["br_sz"]


def test_all_residuals_zero_and_constant_field():
    """Residuals all zero: b = 1, one bin, entropy 0, MSE of the central bin
    (2 u)^2 / 12.  A constant field: flagged, nothing estimated."""
    r = O.estimate_sz_log(np.ones(8, np.float32), O.params())
    assert r["flags"] & O.F_CONSTANT and math.isinf(r["psnr_log"])
    z = np.zeros(32, np.float32)
    z[0] = 7.0  # residual 7 then -7 then zeros: value range 7
    r = O.estimate_sz_log(z, O.params(eb=1.0, eb_mode=O.EB_ABS, r_sp=1.0, quant_radius=4),
                          want_hist=True)
    assert r["max_abs"] == 7.0 and r["base"] > 1.0
    w = np.zeros(32, np.float32) + 2.0
    w[16:] = 3.0  # residuals 2, 0.., 1, 0..: max 2
    r = O.estimate_sz_log(w, O.params(eb=4.0, eb_mode=O.EB_ABS, r_sp=1.0), want_hist=True)
    assert r["base"] == 1.0 and r["hist"][32768] == 32 and r["entropy"] == 0.0
    assert r["mse_log"] == (2 * 4.0) ** 2 / 12
