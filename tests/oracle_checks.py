"""Checks of the oracle's SZ quantisers and entropy against their plain
definitions, shared by the pins (test_oracle_definitions.py) and by the
planted-mutation tests (test_oracle_mutations.py), which run the same checks
on deliberately broken builds of the oracle and expect them to fail.

Each check takes the oracle module (whose library may be a mutant) and raises
AssertionError when the oracle departs from the definition:

  entropy    Eq. (entropy) with Eq. (bitrate-sz) for linear bins: the bit-rate
             is -sum p log2 p over the bin frequencies p = h / N_s, plus the
             0.5-bit offset of the evaluation section;
  estimator  Section "Estimation Based on Static Quantization", linear case:
             the code of a sampled point is q = floor(r / delta + 0.5) with
             r = x - pred, pred the Lorenzo prediction from the original
             neighbours (Section "Prediction-Based Transformation"), zero
             outside the field;
  truth      the prequantised code Q = floor(x / delta + 0.5) and its
             reconstruction Q * delta.

The oracle takes the quantisation decision in float32 (the precision the
GPU path computes in): the residual as nested float32 differences, the code
as rint(r * (1/w)) with w = float(delta) and 1/w rounded to float.  The
checks therefore allow a code to differ from the float64 definition by one,
and only where the float64 value r / delta lies within the float32 rounding
error of a bin edge (k + 1/2); the error bound is derived below.
"""
from __future__ import annotations

import math

import numpy as np

EPS32 = 2.0 ** -24  # unit roundoff of float32


def lorenzo_residual_f64(x: np.ndarray) -> np.ndarray:
    """x - pred in float64, zero outside the field: the mixed first
    difference along every axis (the Lorenzo predictor of 1/3/7 preceding
    neighbours makes x - pred the sum over axis subsets S of
    (-1)^|S| x(idx - e_S))."""
    r = x.astype(np.float64)
    for ax in range(x.ndim):
        r = np.diff(r, axis=ax, prepend=0.0)
    return r


def stencil_abs_sum(x: np.ndarray) -> np.ndarray:
    """Sum of |x| over each point's 2^d stencil points (zero outside)."""
    m = np.abs(x.astype(np.float64))
    for ax in range(x.ndim):
        pad = [(0, 0)] * x.ndim
        pad[ax] = (1, 0)
        sl = [slice(None)] * x.ndim
        sl[ax] = slice(0, -1)
        m = m + np.pad(m, pad)[tuple(sl)]
    return m


def _edge_distance(t: np.ndarray) -> np.ndarray:
    """Distance of t from the nearest bin edge k + 1/2."""
    return np.abs(t - (np.floor(t) + 0.5))


def _band_estimator(t: np.ndarray, m: np.ndarray, delta: float, d: int) -> np.ndarray:
    """Bound on |rint-argument - r/delta| of the float32 evaluation: the
    2^d - 1 nested differences each round once, with error at most
    EPS32 times their magnitude, itself at most the stencil's sum of |x|
    (m); the product r32 * fl(1/fl(delta)) carries three more relative
    roundings.  Doubled as a margin."""
    return 2.0 * (((1 << d) - 1) * EPS32 * m / delta * (1 + 4 * EPS32) + 3.01 * EPS32 * np.abs(t))


def estimator_disagreements(O, x: np.ndarray, delta: float, radius: int = 32768) -> dict:
    """Every sampled point's code (strides 1: every block sampled) against
    floor(r / delta + 0.5) in float64.  Returns the counts."""
    d = x.ndim
    s = O.sz_symbols(x, delta, quant_radius=radius, strides=[1] * d)
    sym = s["est"].astype(np.int64)
    assert np.all(sym >= 0), "every point of a fully sampled field has a code"
    r = lorenzo_residual_f64(x)
    t = r / delta
    qdef = np.floor(t + 0.5)
    esc_def = np.abs(qdef) >= radius
    q = sym - 32768
    band = _band_estimator(t, stencil_abs_sum(x), delta, d)
    near = _edge_distance(t) <= band
    # escapes: symbol 0 exactly when |q| >= R (up to a code at the edge)
    esc = sym == 0
    bad_esc = esc != esc_def
    assert not np.any(bad_esc & ~near), "escape decisions away from a bin edge differ"
    both = ~esc & ~esc_def
    diff = q[both] - qdef[both]
    assert np.all(np.abs(diff) <= 1), "a code differs by more than one bin"
    off = diff != 0
    assert not np.any(off & ~near[both]), (
        "codes away from a bin edge differ from floor(r/delta + 0.5)",
        int(np.count_nonzero(off & ~near[both])))
    return {"points": int(sym.size), "differ": int(np.count_nonzero(off)),
            "near_edge": int(np.count_nonzero(near)), "escapes": int(np.count_nonzero(esc))}


def truth_disagreements(O, x: np.ndarray, delta: float, radius: int = 32768) -> dict:
    """The ground truth against the definition: prequantised codes
    Q = floor(x / delta + 0.5) in float64, residual codes the integer Lorenzo
    residual of Q (zero outside), a point escaping when its residual code
    reaches the radius.  The oracle's codes are recovered from the
    reconstruction of the points that did not escape (recon = float(Q) * w,
    so recon / w = Q to within Q * 2^-23).  The float32 decision may differ
    from the definition only at points within rounding of a bin edge, and an
    escape or a residual code only where its stencil holds such a point (a
    reconstruction error within rounding of delta / 2 also escapes)."""
    s = O.sz_symbols(x, delta, quant_radius=radius)
    gt = s["gt"].astype(np.int64)
    esc = gt == 0
    t = x.astype(np.float64) / delta
    qdef = np.floor(t + 0.5).astype(np.int64)
    res = qdef
    for ax in range(x.ndim):
        res = np.diff(res, axis=ax, prepend=0)
    esc_def = np.abs(res) >= radius
    band = 2.0 * 3.01 * EPS32 * np.abs(t)
    near = _edge_distance(t) <= band
    near_st = stencil_abs_sum(near.astype(np.float32)) > 0
    assert not np.any((esc != esc_def) & ~near_st), (
        "escapes away from a bin edge differ from |residual| >= R",
        int(np.count_nonzero((esc != esc_def) & ~near_st)))
    w = float(np.float32(delta))
    y = s["recon"].astype(np.float64) / w
    qrec = np.rint(y)
    ok = ~esc
    # the reconstruction is a whole number of bins
    assert np.all(np.abs(y[ok] - qrec[ok]) <= np.abs(qrec[ok]) * 2.0 ** -22 + 1e-9), (
        "reconstruction is not float(Q) * w for an integer Q")
    diff = qrec[ok] - qdef[ok]
    assert np.all(np.abs(diff) <= 1), "a prequantised code differs by more than one bin"
    off = diff != 0
    assert not np.any(off & ~near[ok]), (
        "prequantised codes away from a bin edge differ from floor(x/delta + 0.5)",
        int(np.count_nonzero(off & ~near[ok])))
    clean = ok & ~near_st
    assert np.array_equal(gt[clean], res[clean] + 32768), "residual codes differ"
    return {"points": int(x.size), "differ": int(np.count_nonzero(off)),
            "near_edge": int(np.count_nonzero(near)), "escapes": int(np.count_nonzero(esc))}


def _ramp_field(codes: np.ndarray) -> np.ndarray:
    """A 1D field whose Lorenzo residuals at bin width 1 are exactly `codes`:
    their running sum (integers, exact in float32 below 2^24)."""
    x = np.cumsum(codes.astype(np.int64))
    assert np.abs(x).max() < 2 ** 24
    return x.astype(np.float32)


def check_entropy_equal_bins(O):
    """Equal counts over 2^k codes: the histogram is known, the entropy is
    exactly k bits and BR_sz = k + 0.5 exactly (every term is dyadic)."""
    for k in (1, 3, 8, 12):
        n = 1 << 14
        codes = (np.arange(n) % (1 << k)) - (1 << (k - 1))
        x = _ramp_field(codes)
        r = O.estimate_sz(x, O.params(eb=1e-3, r_sp=1.0), delta=1.0, want_hist=True)
        h = r["hist"]
        assert int(h.sum()) == n and r["sz_ns"] == n
        assert np.count_nonzero(h) == 1 << k
        assert np.all(h[h > 0] == n >> k)
        assert r["entropy"] == float(k), (k, r["entropy"])
        assert r["br_sz"] == k + 0.5, (k, r["br_sz"])


def check_entropy_unequal_bins(O):
    """A known unequal histogram (rounded normal codes): the entropy equals
    -sum p log2 p summed exactly (math.fsum) to 1e-14 relative, and so does
    BR_sz - 0.5."""
    rng = np.random.default_rng(77)
    codes = np.rint(rng.standard_normal(1 << 14) * 6.0).astype(np.int64)
    x = _ramp_field(codes)
    r = O.estimate_sz(x, O.params(eb=1e-3, r_sp=1.0), delta=1.0, want_hist=True)
    h = r["hist"].astype(np.int64)
    ref_h = np.bincount(codes + 32768, minlength=65536)
    assert np.array_equal(h, ref_h), "histogram of the known codes"
    n = int(h.sum())
    H = -math.fsum((v / n) * math.log2(v / n) for v in h[h > 0])
    assert abs(r["entropy"] - H) <= 1e-14 * H, (r["entropy"], H)
    assert abs((r["br_sz"] - 0.5) - H) <= 1e-14 * H, (r["br_sz"], H)


def check_log_bins_and_mse(O):
    """Log-scale estimate on known residuals (a skewed, mostly positive set):
    every residual's code against the exact edges u b^k (rationals) away
    from rounding of an edge, and the MSE of Eq. (mse-pdf) summed exactly."""
    from fractions import Fraction

    rng = np.random.default_rng(91)
    codes = np.rint(np.abs(rng.standard_normal(3000)) * 400 - 40).astype(np.int64)
    x = _ramp_field(codes)
    n = 64
    p = O.params(eb=0.5, eb_mode=1, r_sp=1.0, quant_radius=n)
    r = O.estimate_sz_log(x, p, want_hist=True, want_edges=True)
    u, b = Fraction(r["unit"]), Fraction(r["base"])
    exact = [u]
    for _ in range(n):
        exact.append(exact[-1] * b)
    want = np.zeros(65536, np.int64)
    near = 0
    for c in codes:
        a = Fraction(abs(int(c)))
        k = sum(1 for j in range(1, n) if exact[j] <= a)
        near += any(abs(a - exact[j]) <= a * Fraction(1, 2 ** 48) for j in range(1, n))
        want[32768 + (k if c >= 0 else -k)] += 1
    got = r["hist"].astype(np.int64)
    assert np.abs(got - want).sum() <= 2 * near, "codes differ from the exact bins"
    A = [r["unit"]] + list(r["edges"])
    tot = Fraction(0)
    for s in np.nonzero(got)[0]:
        k = abs(int(s) - 32768)
        w = Fraction(2 * A[1]) if k == 0 else Fraction(A[k + 1]) - Fraction(A[k])
        tot += int(got[s]) * w * w
    mse = tot / (12 * int(got.sum()))
    assert abs(Fraction(r["mse_log"]) - mse) <= mse * Fraction(1, 10 ** 13), "MSE of the bins"
