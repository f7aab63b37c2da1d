"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
values the paper prints (tests/golden/), closed forms, invariants, special
cases that reduce to a library routine, and brute force on tiny inputs.  They
run without a GPU.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
import synth

O = pytest.importorskip("oracle")


def _golden_dict(name):
    return {r[0]: r[1:] for r in read_golden(name)}


# ---------------------------------------------------------------------------
# Algorithm 1 line 2: value range
# ---------------------------------------------------------------------------

def test_value_range_matches_numpy():
    x = synth.config1_field(seed=11, shape=(37, 53))
    r = O.select(x, O.params(eb=1e-3, r_sp=1.0))
    assert r["vmin"] == np.float32(x.min()) and r["vmax"] == np.float32(x.max())
    assert r["vr"] == float(x.max()) - float(x.min())
    assert r["eb_abs"] == 1e-3 * r["vr"]
    # minexp = floor(log2 eb_abs), checked against math.log2 on a non-power
    assert r["minexp"] == math.floor(math.log2(r["eb_abs"]))


def test_constant_field_and_nonfinite():
    x = np.full((9, 10), 3.5, np.float32)
    r = O.select(x, O.params())
    assert r["flags"] & O.F_CONSTANT and r["selection"] == 1
    assert math.isinf(r["psnr_zfp"]) and r["br_zfp"] == 0.0
    y = np.zeros((8, 8), np.float32)
    y[3, 4] = np.nan
    with pytest.raises(O.OracleError) as e:
        O.select(y, O.params())
    assert e.value.code == O.ERR_NONFINITE
    y[3, 4] = np.inf
    with pytest.raises(O.OracleError):
        O.ground_truth(y, O.params())


# ---------------------------------------------------------------------------
# Sampling (Sec. "Data Sampling"; reading: prime-factor strides)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,r_sp,strides", [
    ((100, 500, 500), 0.05, [2, 2, 5]),
    ((100, 500, 500), 0.01, [4, 5, 5]),
    ((1800, 3600), 0.05, [4, 5]),
    ((1800, 3600), 0.01, [10, 10]),
    ((4096,), 0.05, [20]),
    ((64, 64), 1.0, [1, 1]),
])
def test_sampling_strides_and_counts(shape, r_sp, strides):
    st, nsb, npts = O.sampling(shape, r_sp)
    assert st == strides
    # closed form: per axis ceil(B_k / s_k) sampled blocks, each with
    # min(4, n_k - 4 b) valid points; the lattice is a product over axes
    blocks = [(n + 3) // 4 for n in shape]
    assert nsb == math.prod((b + s - 1) // s for b, s in zip(blocks, st))
    pts = 1
    for n, b, s in zip(shape, blocks, st):
        pts *= sum(min(4, n - 4 * j) for j in range(0, b, s))
    assert npts == pts
    # the sampled fraction is close to the requested rate on large grids
    if math.prod(blocks) >= 10000:
        assert abs(nsb / math.prod(blocks) - r_sp) < 0.25 * r_sp


def test_default_sampling_rate_is_papers():
    g = _golden_dict("paper_constants.txt")
    assert float(g["default_r_sp"][0]) == O.params().r_sp


# ---------------------------------------------------------------------------
# ZFP transform (Sec. "Block Orthogonal Transformation"; zfp publication)
# ---------------------------------------------------------------------------

def _zfp_matrix():
    g = _golden_dict("bot_transforms.txt")
    return np.array([[int(v) for v in g[f"zfp_fwd_row{i}"]] for i in range(4)])


def test_forward_lifting_equals_published_matrix():
    """On inputs where every shift is exact (multiples of 64) the lifting
    scheme computes exactly (1/16) M v with the published matrix M."""
    M = _zfp_matrix()
    rng = np.random.default_rng(5)
    for _ in range(500):
        v = rng.integers(-2 ** 23, 2 ** 23, 4) * 64
        got = O.fwd_lift(v)
        want = [Fraction(int(x), 16) for x in M @ v]
        assert [Fraction(t) for t in got] == want
        assert O.inv_lift(got) == [int(t) for t in v]


def test_inverse_lifting_close_on_arbitrary_inputs():
    rng = np.random.default_rng(6)
    worst = 0
    for _ in range(2000):
        v = rng.integers(-2 ** 29, 2 ** 29, 4)
        back = O.inv_lift(O.fwd_lift(v))
        worst = max(worst, max(abs(a - int(b)) for a, b in zip(back, v)))
    assert worst <= 8


def test_zfp_transform_is_half_an_orthonormal_one():
    """The paper's T(t) is orthonormal (Lemma 1's premise); zfp's matrix is
    close to (1/2) T: each row of 2M/16 has norm within 15% of one.  This is
    why the estimator rescales coefficient errors by 2^d."""
    M = _zfp_matrix() / 16.0
    norms = np.linalg.norm(2.0 * M, axis=1)
    assert np.all(np.abs(norms - 1.0) < 0.15)
    assert not np.allclose((2 * M) @ (2 * M).T, np.eye(4))


def test_zfp_matrix_has_the_parametric_form_at_half_scale():
    """2 x zfp's matrix has the row pattern of T(t) = (1/2)[[1,1,1,1],
    [c,s,-s,-c],[1,-1,-1,1],[s,-c,c,-s]]: rows 0 and 2 are T's (row 2 up to
    sign), rows 1 and 3 follow the (c, s) pattern with c^2 + s^2 = 26/16 and
    40/16 instead of 2.  So one zfp step computes half a T-form coefficient,
    and d steps 2^-d of it: the scale the MSE_sp estimate undoes before
    Theorem 1 applies."""
    M = [[Fraction(int(v), 16) for v in row] for row in _zfp_matrix()]
    T2 = [[2 * v for v in row] for row in M]  # 2 x zfp = (1/2) x pattern
    half = Fraction(1, 2)
    assert T2[0] == [half] * 4
    assert T2[2] == [-half, half, half, -half]
    c, s = 2 * T2[1][0], 2 * T2[1][1]
    assert T2[1] == [c / 2, s / 2, -s / 2, -c / 2] and c * c + s * s == Fraction(26, 16)
    s3, c3 = 2 * T2[3][0], -2 * T2[3][1]
    assert T2[3] == [s3 / 2, -c3 / 2, c3 / 2, -s3 / 2] and c3 * c3 + s3 * s3 == Fraction(40, 16)


def test_bot_orthogonality_and_l2_invariance():
    """Lemma 1 / Theorem 1: T(t) T(t)^T = I for the named transforms, and
    applying T along every axis of a 4^3 block (unfold/fold) preserves the
    elementwise L2 norm."""
    rng = np.random.default_rng(7)
    blk = rng.standard_normal((4, 4, 4))
    for name, vals in _golden_dict("bot_transforms.txt").items():
        if name.startswith("zfp"):
            continue
        t = float(vals[0])
        s, c = math.sqrt(2) * math.sin(math.pi * t / 2), math.sqrt(2) * math.cos(math.pi * t / 2)
        T = 0.5 * np.array([[1, 1, 1, 1], [c, s, -s, -c], [1, -1, -1, 1], [s, -c, c, -s]])
        assert np.allclose(T @ T.T, np.eye(4), atol=1e-12), name
        y = blk
        for ax in range(3):
            y = np.moveaxis(np.tensordot(T, np.moveaxis(y, ax, 0), axes=1), 0, ax)
        assert abs(np.linalg.norm(y) - np.linalg.norm(blk)) < 1e-12


def test_negabinary_against_base_minus_two_digits():
    """u = (i + M) xor M must be the base(-2) digit string of i."""
    rng = np.random.default_rng(8)
    vals = list(range(-40, 41)) + [int(v) for v in rng.integers(-2 ** 30, 2 ** 30, 500)]
    for i in vals:
        u = O.int2nb(i)
        assert sum(((u >> k) & 1) * (-2) ** k for k in range(32)) == i
        assert O.nb2int(u) == i
    # a few worked values: 1 -> 1, -1 -> 0b11, 2 -> 0b110, -2 -> 0b10, 3 -> 0b111
    assert [O.int2nb(i) for i in (1, -1, 2, -2, 3)] == [1, 3, 6, 2, 7]


def test_sequency_order_properties():
    for d in (1, 2, 3):
        perm = O.sequency(d)
        assert sorted(perm) == list(range(4 ** d)) and perm[0] == 0
        tuples = [tuple((t >> (2 * (d - 1 - k))) & 3 for k in range(d)) for t in perm]
        sums = [sum(t) for t in tuples]
        assert sums == sorted(sums)
        # the last coefficient is the highest-frequency one (3, ..., 3)
        assert tuples[-1] == (3,) * d


@pytest.mark.parametrize("d", [1, 2, 3])
def test_constant_block_is_dc_only(d):
    for c in (1.0, -0.37, 3.0e-30, 1.5e20, 2.0 ** -130):
        v = np.full(4 ** d, c, np.float32)
        o = O.zfp_block(v, d, minexp=-30)
        e = math.frexp(float(np.float32(c)))[1]
        e = max(e, -126)
        assert o["emax"] == e
        dc = int(Fraction(float(np.float32(c))) * Fraction(2) ** (30 - e))
        assert o["coeff_int"][0] == dc
        assert all(t == 0 for t in o["coeff_int"][1:])


@pytest.mark.parametrize("d", [1, 2, 3])
def test_block_exponent_and_cast_exact(d):
    rng = np.random.default_rng(9 + d)
    for _ in range(50):
        v = (rng.standard_normal(4 ** d) * 10.0 ** rng.integers(-30, 30)).astype(np.float32)
        o = O.zfp_block(v, d, minexp=-40)
        emax = max(max(math.frexp(float(t))[1], -126) for t in v if t != 0)
        assert o["emax"] == emax
        assert o["prec"] == min(32, max(0, emax + 40 + 2 * (d + 1)))


# ---------------------------------------------------------------------------
# Embedded coding bits (Sec. "Estimation Based on Dynamic Quantization")
# ---------------------------------------------------------------------------

def _group_test_bits(u, kmin):
    """Brute-force group-testing emitter written from its description: emit
    the verbatim bits of the significant prefix, then test the rest for a
    one, scanning bit by bit to it (the last position's one is implied)."""
    nb = len(u)
    n, bits = 0, 0
    for k in range(31, kmin - 1, -1):
        plane = [(w >> k) & 1 for w in u]
        bits += n
        i = n
        while i < nb:
            bits += 1
            if not any(plane[i:]):
                break
            while True:
                if i == nb - 1:
                    break
                bits += 1
                if plane[i]:
                    break
                i += 1
            i += 1
            n = i
    return bits


@pytest.mark.parametrize("d", [1, 2, 3])
def test_embedded_coding_bits_three_ways(d):
    rng = np.random.default_rng(20 + d)
    for trial in range(60):
        scale = 10.0 ** rng.integers(-3, 4)
        v = (rng.standard_normal(4 ** d) * scale).astype(np.float32)
        if trial % 5 == 0:
            v[: rng.integers(1, 4 ** d)] = 0
        minexp = int(rng.integers(-30, 5))
        o = O.zfp_block(v, d, minexp)
        assert o["bits_emitter"] == o["bits_closed"]
        if o["prec"] == 0:
            assert o["bits_closed"] == 1
        else:
            assert o["bits_closed"] == 9 + _group_test_bits(o["coeff_nb"], o["kmin"])


def test_empty_and_fill_blocks_cost_one_bit():
    o = O.zfp_block(np.zeros(16, np.float32), 2, minexp=-20)
    assert o["all_zero"] and o["prec"] == 0 and o["bits_closed"] == 1
    # 1e-20 fill values under an error bound of 1e-5 of a unit range: P = 0
    o = O.zfp_block(np.full(64, 1e-20, np.float32), 3, minexp=math.floor(math.log2(1e-5)))
    assert o["prec"] == 0 and o["bits_closed"] == 1


def test_ec_positions_counts_from_paper():
    g = _golden_dict("paper_constants.txt")
    for d, key in ((1, "ec_samples_1d"), (2, "ec_samples_2d"), (3, "ec_samples_3d")):
        pos = O.ec_positions(d)
        assert len(pos) == int(g[key][0])
        assert pos[0] == 0 and pos[-1] == 4 ** d - 1 and pos == sorted(set(pos))
        assert O.ec_positions(d, O.EC_ALL) == list(range(4 ** d))
    assert O.ec_positions(2) == [0, 2, 4, 6, 8, 9, 11, 13, 15]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_interpolated_nsb_sum(d):
    """Doubled sum of the piecewise-linear interpolation through the sampled
    n_sb equals twice the explicit sum of interpolated values; under EC_ALL it
    is exactly 2 sum(n_sb)."""
    rng = np.random.default_rng(30 + d)
    for _ in range(30):
        v = (rng.standard_normal(4 ** d) * 100).astype(np.float32)
        o = O.zfp_block(v, d, minexp=-12)
        pos = O.ec_positions(d)
        nsb = o["nsb"]
        total = Fraction(0)
        for p in range(4 ** d):
            j = max(i for i in range(len(pos)) if pos[i] <= p)
            if pos[j] == p:
                total += nsb[p]
            else:
                a, b = pos[j], pos[j + 1]
                total += nsb[a] + Fraction(nsb[b] - nsb[a], b - a) * (p - a)
        assert o["s2_block"] == 2 * total
        oa = O.zfp_block(v, d, minexp=-12, ec_mode=O.EC_ALL)
        assert oa["s2_block"] == 2 * sum(oa["nsb"])


def test_nsb_counts_planes_from_leading_one():
    rng = np.random.default_rng(40)
    v = (rng.standard_normal(16) * 7).astype(np.float32)
    o = O.zfp_block(v, 2, minexp=-10)
    for u, n in zip(o["coeff_nb"], o["nsb"]):
        top = u.bit_length() - 1
        assert n == (top - o["kmin"] + 1 if top >= o["kmin"] else 0)


@pytest.mark.parametrize("d,shape", [(1, (1001,)), (2, (61, 58)), (3, (17, 22, 19))])
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_zfp_error_bound_holds(d, shape, eb):
    """Fixed-accuracy ZFP keeps |x - xhat| <= eb_abs at every point: this pins
    the precision rule, the transform pair and the reconstruction together."""
    x = synth.grf_np(shape, -3.0, seed=100 + d).astype(np.float32) * 40.0
    t = O.ground_truth(x, O.params(eb=eb, r_sp=1.0))
    r = O.select(x, O.params(eb=eb, r_sp=1.0))
    assert t["maxerr_zfp"] <= r["eb_abs"]


# ---------------------------------------------------------------------------
# Exact MSE, delta and PSNR (Eqs. psnr-pdf, psnr-pdf-linear, psnr-sz)
# ---------------------------------------------------------------------------

def test_mse_numerator_is_exact_sum_rounded_once():
    rng = np.random.default_rng(50)
    for _ in range(40):
        n = int(rng.integers(1, 200))
        e = rng.integers(-126, 132, n).astype(np.int32)
        e[: n // 2] = e[0]  # shared exponents exercise carries
        dd = rng.integers(-2 ** 32 + 1, 2 ** 32, n, dtype=np.int64)
        exact = sum(Fraction(int(a)) ** 2 * Fraction(4) ** (int(b) - 30) for a, b in zip(dd, e))
        assert O.mse_numerator(e, dd) == float(exact)


def test_delta_matches_psnr_equality():
    """Alg. 1 line 7: with PSNR_sz = PSNR_zfp in Eq. (psnr-pdf-linear), VR
    cancels and delta^2 = 12 MSE_sp."""
    x = synth.config1_field(seed=3, shape=(96, 80))
    for eb in (1e-2, 1e-3, 1e-4):
        r = O.select(x, O.params(eb=eb, r_sp=0.25))
        if r["flags"] & (O.F_DELTA_CLAMPED | O.F_MSE_ZERO):
            continue
        psnr_linear = 20 * math.log10(r["vr"] / r["delta"]) + 10 * math.log10(12)
        assert abs(psnr_linear - r["psnr_zfp"]) < 1e-9 * abs(r["psnr_zfp"])
        assert r["psnr_sz"] == pytest.approx(r["psnr_zfp"], rel=1e-12)


def test_psnr_sz_closed_form_when_delta_is_twice_eb():
    """Eq. (psnr-sz): with delta = 2 eb_abs, PSNR_sz = -20 log10(eb_rel) +
    10 log10 3."""
    x = np.linspace(0, 1, 4096, dtype=np.float32).reshape(64, 64)
    for eb in (1e-2, 1e-3, 1e-4):
        r = O.select(x, O.params(eb=eb, r_sp=1.0))
        if not r["flags"] & (O.F_DELTA_CLAMPED | O.F_MSE_ZERO):
            continue
        want = -20 * math.log10(eb) + 10 * math.log10(3)
        assert r["psnr_sz"] == pytest.approx(want, rel=1e-12)


def test_mse_sp_from_exported_coefficients():
    """MSE_sp equals the exact mean of (2^d d)^2 4^(emax-30) over the
    EC-sampled coefficients of the sampled blocks, recomputed from per-block
    oracle records with Python integers."""
    x = synth.config1_field(seed=4, shape=(40, 36))
    p = O.params(eb=1e-3, r_sp=0.25)
    r = O.select(x, p)
    st = r["strides"]
    pos = O.ec_positions(2)
    acc, cnt = Fraction(0), 0
    for by in range(0, 10, st[0]):
        for bx in range(0, 9, st[1]):
            blk = x[4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
            o = O.zfp_block(blk, 2, r["minexp"])
            for j in pos:
                if not o["all_zero"]:
                    acc += Fraction(o["d"][j]) ** 2 * Fraction(4) ** (o["emax"] + 2 - 30)
                cnt += 1
    assert cnt == r["zfp_ncoeff"]
    assert r["mse_sp"] == float(acc) / cnt


# ---------------------------------------------------------------------------
# SZ estimator and ground truth (Sec. PBT, Eq. bitrate-sz, Eq. entropy)
# ---------------------------------------------------------------------------

def _multilinear(shape, rng):
    """Integer field that is at most linear in each coordinate separately and
    has no product of all axes: every mixed difference over all axes is 0."""
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    f = np.full(shape, int(rng.integers(-5, 5)), np.int64)
    for g in grids:
        f += int(rng.integers(-3, 4)) * g
    if len(shape) == 3:  # pairwise products are not products of all axes
        for a, b in itertools.combinations(range(3), 2):
            f += int(rng.integers(-2, 3)) * grids[a] * grids[b]
    return f.astype(np.float32)


@pytest.mark.parametrize("shape", [(50,), (13, 17), (6, 7, 9)])
def test_lorenzo_exact_on_multilinear_fields(shape):
    """The Lorenzo predictor reproduces multilinear data exactly, so interior
    points (every coordinate >= 1) get code 0 (symbol 32768)."""
    x = _multilinear(shape, np.random.default_rng(len(shape)))
    s = O.sz_symbols(x, delta=0.5, strides=[1, 1, 1][: len(shape)])
    interior = tuple(slice(1, None) for _ in shape)
    assert np.all(s["est"][interior] == 32768)


@pytest.mark.parametrize("shape", [(64,), (12, 15), (5, 6, 7)])
def test_gt_codes_are_integer_lorenzo_residuals(shape):
    """Integer-valued field with delta = 1: prequantisation is the identity
    and the ground-truth codes are the mixed first differences of the data
    with zero padding, computed here with numpy's diff."""
    rng = np.random.default_rng(60 + len(shape))
    x = rng.integers(-50, 50, shape).astype(np.float32)
    s = O.sz_symbols(x, delta=1.0)
    r = x.astype(np.int64)
    for ax in range(len(shape)):
        r = np.diff(r, axis=ax, prepend=0)
    assert np.array_equal(s["gt"], (r + 32768).astype(np.int32))
    assert np.array_equal(s["recon"], x)


@pytest.mark.parametrize("shape", [(997,), (41, 39), (11, 13, 17)])
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_sz_gt_error_bound_holds(shape, eb):
    x = (synth.grf_np(shape, -3.0, seed=200 + len(shape)) * 25 + 100).astype(np.float32)
    r = O.select(x, O.params(eb=eb, r_sp=1.0))
    t = O.ground_truth(x, O.params(eb=eb, r_sp=1.0))
    assert t["eb_sz"] == r["delta"] / 2
    assert t["maxerr_sz"] <= t["eb_sz"]
    # the reconstruction is recomputed in float64 from the exported recon
    s = O.sz_symbols(x, delta=r["delta"])
    err = np.abs(x.astype(np.float64) - s["recon"].astype(np.float64))
    assert err.max() == t["maxerr_sz"]
    assert np.count_nonzero(s["gt"] == 0) == t["sz_nesc_gt"]


def test_escape_when_code_exceeds_radius():
    x = np.array([0, 0, 0, 100, 0, 0], np.float32)
    s = O.sz_symbols(x, delta=1.0, quant_radius=10)
    # residuals: 0 0 0 100 -100 0 -> the two large ones escape (symbol 0)
    assert list(s["gt"]) == [32768, 32768, 32768, 0, 0, 32768]
    assert np.array_equal(s["recon"], x)


def test_estimator_histogram_counts_sampled_points():
    x = synth.config1_field(seed=6, shape=(50, 45))
    r = O.select(x, O.params(eb=1e-3, r_sp=0.05), want_hist=True)
    assert int(r["hist"].sum()) == r["sz_ns"] == r["zfp_npoints"]
    s = O.sz_symbols(x, delta=r["delta"], strides=r["strides"])
    est = s["est"][s["est"] >= 0]
    assert np.array_equal(np.bincount(est, minlength=65536), r["hist"])


# ---------------------------------------------------------------------------
# Huffman cost and entropy (Stage III)
# ---------------------------------------------------------------------------

def _brute_force_prefix_cost(w):
    """Minimum total cost over every order of pairwise merges: every binary
    prefix code tree is reachable this way, so this is the optimum."""
    best = [None]

    def rec(items, acc):
        if len(items) == 1:
            if best[0] is None or acc < best[0]:
                best[0] = acc
            return
        for i, j in itertools.combinations(range(len(items)), 2):
            s = items[i] + items[j]
            rest = [items[k] for k in range(len(items)) if k not in (i, j)] + [s]
            rec(rest, acc + s)

    rec(list(w), 0)
    return best[0]


def test_huffman_textbook_values():
    for row in read_golden("huffman_textbook.txt"):
        k = row.index("=")
        assert O.huffman_cost([int(v) for v in row[:k]]) == int(row[k + 1])


def test_huffman_brute_force_and_bounds():
    rng = np.random.default_rng(70)
    for K in range(2, 7):
        for _ in range(6):
            w = [int(v) for v in rng.integers(1, 50, K)]
            c = O.huffman_cost(w)
            assert c == _brute_force_prefix_cost(w)
            n = sum(w)
            H = -sum(v / n * math.log2(v / n) for v in w)
            assert H * n <= c + 1e-9 and c < (H + 1) * n
            # tie order / input order do not change the total
            assert O.huffman_cost(list(rng.permutation(w))) == c
            assert O.huffman_cost([0] + w + [0, 0]) == c


def test_huffman_special_cases():
    assert O.huffman_cost([0, 0, 0]) == 0
    assert O.huffman_cost([0, 17, 0]) == 17
    for k in range(1, 9):
        assert O.huffman_cost([5] * 2 ** k) == k * 5 * 2 ** k


def test_entropy_of_equal_bins_and_offset():
    """Equal counts over 2^k bins: entropy exactly k; BR_sz = H + 0.5."""
    x = np.tile(np.arange(8, dtype=np.float32), 8 * 64)  # 1D ramp of period 8
    r = O.select(x, O.params(eb=1e-4, r_sp=1.0, eb_mode=O.EB_REL))
    assert r["br_sz"] == pytest.approx(r["entropy"] + 0.5, abs=0)
    g = _golden_dict("paper_constants.txt")
    assert float(g["sz_offset_bits"][0]) == O.params().sz_offset
    h = np.zeros(65536, np.uint32)
    h[100:116] = 7
    n = int(h.sum())
    H = -sum(v / n * math.log2(v / n) for v in h[h > 0])
    assert H == pytest.approx(4.0, abs=1e-15)


def test_histogram_alphabet_matches_paper_bins():
    """n_pdf = 65535 bins (2n-1 with n = 32768) plus one escape symbol, and the
    memory-overhead figures of the paper follow from it."""
    g = _golden_dict("paper_constants.txt")
    assert int(g["n_pdf_bins"][0]) + 1 == O.NSYM
    for pts, pct in (("atm_points", "atm_mem_overhead_pct"),
                     ("hurricane_points", "hurricane_mem_overhead_pct")):
        ov = 100.0 * int(g["n_pdf_bins"][0]) / int(g[pts][0])
        assert abs(ov - float(g[pct][0])) < 0.06


# ---------------------------------------------------------------------------
# Selection (Alg. 1 lines 10-12)
# ---------------------------------------------------------------------------

def test_selection_follows_estimated_rates():
    rng = np.random.default_rng(80)
    smooth = synth.config1_field(seed=8, shape=(128, 128))
    noisy = rng.standard_normal((128, 128)).astype(np.float32)
    for x in (smooth, noisy):
        for eb in (1e-2, 1e-3, 1e-4):
            r = O.select(x, O.params(eb=eb, r_sp=0.25))
            if r["flags"] & O.F_TIE_BAND:
                assert r["selection"] == 1
            else:
                assert r["selection"] == (0 if r["br_sz"] < r["br_zfp"] else 1)
            rh = O.select(x, O.params(eb=eb, r_sp=0.25, sel_rule=O.SEL_HUFFMAN))
            lhs = Fraction(rh["sz_huff_bits"] + 32 * rh["sz_nesc"], rh["sz_ns"])
            rhs = Fraction(rh["zfp_s2"], 2 * rh["zfp_npoints"])
            assert rh["selection"] == (0 if lhs < rhs else 1)


def test_ratios_are_reasonable_on_smooth_field():
    """A smooth 2D field compresses to few bits/value; both estimates and the
    ground truth agree on the order of magnitude."""
    x = synth.config1_field(seed=9, shape=(128, 128))
    p = O.params(eb=1e-3, r_sp=1.0)
    r = O.select(x, p)
    t = O.ground_truth(x, p)
    assert 0 < r["br_zfp"] < 12 and 0 < r["br_sz"] < 12
    assert abs(r["psnr_zfp"] - t["psnr_zfp_gt"]) < 0.1 * t["psnr_zfp_gt"]
    assert abs(r["psnr_sz"] - t["psnr_sz_gt"]) < 0.1 * t["psnr_sz_gt"]


def test_estimate_sz_agrees_with_select_and_closed_form():
    """rdo_estimate_sz at select's delta reproduces select's SZ fields; at
    delta = 2 eb_abs its PSNR is Eq. (psnr-sz)."""
    x = synth.config1_field(seed=12, shape=(60, 52))
    p = O.params(eb=1e-3, r_sp=0.1)
    r = O.select(x, p, want_hist=True)
    e = O.estimate_sz(x, p, delta=r["delta"], want_hist=True)
    for k in ("sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz", "entropy", "br_sz_huff",
              "psnr_sz", "strides", "zfp_npoints", "n_sampled_blocks"):
        assert e[k] == r[k], k
    assert np.array_equal(e["hist"], r["hist"])
    e2 = O.estimate_sz(x, p, delta=0.0)
    assert e2["delta"] == 2 * e2["eb_abs"]
    assert e2["psnr_sz"] == pytest.approx(-20 * math.log10(1e-3) + 10 * math.log10(3), rel=1e-12)


def test_rd_curve_fixed_error_selection_follows_the_paper():
    """Evaluation section, fixed-PSNR vs fixed-maximum-error selection
    (Fig. f9): at the same maximum error (eb_abs = 1e-3 of the value range)
    the selection based on error bound picks SZ on smooth fields, by
    estimate and by ground truth, while ZFP over-preserves the error (a
    higher PSNR than SZ at the same bound); both stay within eb_abs.  The
    rate-distortion selection is the one of Algorithm 1 at each bound."""
    for x in (synth.config1_field(), synth.config2_field(seed=14, shape=(24, 40, 44))):
        p = O.params(eb=1.0, r_sp=1.0)
        (pt,) = O.rd_curve(x, p, [1e-3])
        assert pt["selection_eb"] == 0 and pt["best_eb_gt"] == 0
        t = pt["truth_eb"]
        assert t["psnr_zfp_gt"] > t["psnr_sz_gt"]
        assert t["maxerr_zfp"] <= pt["est"]["eb_abs"] and t["maxerr_sz"] <= pt["est"]["eb_abs"]
        assert t["eb_sz"] == pt["est"]["eb_abs"]
        assert pt["est_eb"]["delta"] == 2 * pt["est"]["eb_abs"]
        assert pt["est"] == O.select(x, O.params(eb=1e-3, r_sp=1.0))


def _lorenzo_decode(sym, x, w):
    """Decompression of a classic SZ stream written independently of the
    oracle: each value is the Lorenzo prediction from the already decoded
    neighbours (textbook stencil: 1D x[i-1]; 2D x[i,j-1] + x[i-1,j] -
    x[i-1,j-1]; 3D the seven-term inclusion-exclusion) plus its code times
    the bin, or the stored value where the code escaped."""
    d = x.ndim
    xs = np.zeros(x.shape, dtype=np.float64)
    for idx in np.ndindex(*x.shape):
        pred = 0.0
        for sub in range(1, 1 << d):
            off = [(sub >> (d - 1 - k)) & 1 for k in range(d)]
            j = tuple(i - o for i, o in zip(idx, off))
            if min(j) < 0:
                continue
            pred += (1.0 if sum(off) % 2 else -1.0) * xs[j]
        s = int(sym[idx])
        xs[idx] = x[idx] if s == 0 else pred + (s - 32768) * w
    return xs


@pytest.mark.parametrize("shape", [(57,), (9, 13), (5, 6, 7)])
def test_classic_sz_stream_decodes_and_bounds(shape):
    """Classic SZ (prediction from reconstructed neighbours): an independent
    decoder reproduces the oracle's reconstruction from its codes and the
    escaped values (to rounding), every point is within eb_sz, and the
    histogram counts the codes."""
    rng = np.random.default_rng(31)
    x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(np.float32)
    eb_sz = 0.05
    t = O.classic_sz(x, O.params(eb=1e-3, quant_radius=8), eb_sz, want_hist=True,
                     want_recon=True, want_sym=True)
    w = np.float32(2 * eb_sz)
    dec = _lorenzo_decode(t["sym"], x, float(w))
    assert np.max(np.abs(dec - t["recon"].astype(np.float64))) < 1e-4
    assert np.all(np.abs(x.astype(np.float64) - t["recon"]) <= eb_sz)
    assert t["maxerr_sz"] <= eb_sz
    assert np.array_equal(np.bincount(t["sym"].ravel(), minlength=65536), t["hist"])
    assert t["sz_nesc_gt"] == int((t["sym"] == 0).sum()) > 0  # the small radius forces escapes


def test_classic_sz_integer_ramp_closed_form():
    """A 1D integer ramp at bin 1 (eb_sz 0.5): the first point is predicted
    from the zero boundary (code +0), every later one from its exact
    predecessor (code +1), and the reconstruction is exact."""
    x = np.arange(1000, dtype=np.float32)
    t = O.classic_sz(x, O.params(eb=1e-3), 0.5, want_hist=True, want_recon=True)
    h = t["hist"]
    assert h[32768] == 1 and h[32769] == 999 and h.sum() == 1000
    assert np.array_equal(t["recon"], x) and t["maxerr_sz"] == 0.0


def _parse_table(data: bytes):
    """Header and code-length table of an SZ stream, parsed here from the
    bytes (independently of the oracle's decoder)."""
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8))

    def field(pos, nb):
        return int("".join(str(b) for b in bits[pos:pos + nb]), 2), pos + nb

    K, pos = field(0, 32)
    ne, pos = field(pos, 32)
    table = []
    for _ in range(K):
        s, pos = field(pos, 16)
        L, pos = field(pos, 6)
        table.append((s, L))
    return K, ne, table


@pytest.mark.parametrize("shape,radius", [((57,), 8), ((9, 13), 8), ((5, 6, 7), 32768),
                                          ((20, 30), 32768)])
def test_sz_stream_carries_the_classic_truth(shape, radius):
    """The classic truth's bit count is the length of a stream that holds
    everything a decompressor needs: written out (header, code-length table,
    canonical Huffman payload, escaped values), read back symbol for symbol,
    its table a complete prefix code, and the field rebuilt from the stream
    alone by the independent decoder."""
    rng = np.random.default_rng(sum(shape) + radius)
    x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(np.float32)
    eb_sz = 0.05
    t = O.classic_sz(x, O.params(eb=1e-3, quant_radius=radius), eb_sz, want_hist=True,
                     want_recon=True, want_sym=True)
    data, nbits = O.sz_stream(t["sym"], x)
    assert nbits == t["sz_bits_gt"]
    K, ne, table = _parse_table(data)
    assert K == t["sz_nsym_gt"] and ne == t["sz_nesc_gt"]
    assert [s for s, _ in table] == sorted(np.nonzero(t["hist"])[0].tolist())
    if K >= 2:
        assert sum(2.0 ** -L for _, L in table) == 1.0  # Kraft equality: a full tree
    # payload = sum of count x length = the two-queue Huffman cost
    assert sum(int(t["hist"][s]) * L for s, L in table) == t["sz_huff_gt"]
    sym, esc = O.sz_stream_decode(data, nbits, x.size)
    assert np.array_equal(sym, t["sym"].ravel())
    assert np.array_equal(esc.view(np.uint32), x.ravel()[sym == 0].view(np.uint32))
    held = np.full(x.size, np.nan, np.float32)
    held[sym == 0] = esc
    dec = _lorenzo_decode(sym.reshape(shape), held.reshape(shape), float(np.float32(2 * eb_sz)))
    assert np.max(np.abs(dec - t["recon"].astype(np.float64))) < 1e-4


@pytest.mark.parametrize("shape,radius", [((64,), 32768), ((12, 17), 8), ((6, 7, 9), 32768)])
def test_sz_stream_carries_the_prequantised_truth(shape, radius):
    """The same for the prequantised ground truth: the stream of its symbols
    is exactly sz_bits_gt long, and the reconstruction comes back bit for bit
    from the stream alone (integer Lorenzo of the decoded residuals gives
    the codes; an escape's code is that of its stored value)."""
    rng = np.random.default_rng(len(shape) * 7 + radius)
    x = (np.cumsum(rng.standard_normal(shape), axis=-1) * 3).astype(np.float32)
    eb_sz = 0.04
    p = O.params(eb=1e-3, quant_radius=radius)
    t = O.ground_truth(x, p, eb_sz)
    s = O.sz_symbols(x, 2 * eb_sz, quant_radius=radius)
    data, nbits = O.sz_stream(s["gt"], x)
    assert nbits == t["sz_bits_gt"]
    sym, esc = O.sz_stream_decode(data, nbits, x.size)
    assert np.array_equal(sym, s["gt"].ravel())
    w = np.float32(2 * eb_sz)
    inv = np.float32(1.0) / w
    sym = sym.reshape(shape)
    held = np.zeros(x.size, np.float32)
    held[sym.ravel() == 0] = esc
    held = held.reshape(shape)
    d = x.ndim
    Q = np.zeros(shape, dtype=np.int64)
    rec = np.zeros(shape, dtype=np.float32)
    for idx in np.ndindex(*shape):
        if sym[idx] == 0:
            Q[idx] = int(np.rint(np.float32(held[idx] * inv)))
            rec[idx] = held[idx]
            continue
        pred = 0
        for sub in range(1, 1 << d):
            off = [(sub >> (d - 1 - k)) & 1 for k in range(d)]
            j = tuple(i - o for i, o in zip(idx, off))
            if min(j) >= 0:
                pred += (1 if sum(off) % 2 else -1) * int(Q[j])
        Q[idx] = int(sym[idx]) - 32768 + pred
        rec[idx] = np.float32(np.float32(Q[idx]) * w)
    assert np.array_equal(rec.view(np.uint32), s["recon"].view(np.uint32))


def test_sz_stream_single_symbol_and_rejects_bad_streams():
    """One symbol alone costs one bit per point (the cost model's rule);
    a truncated stream or one with bits left over does not parse."""
    x = np.linspace(-1, 1, 100).astype(np.float32)
    sym = np.full(100, 32768, np.int32)
    data, nbits = O.sz_stream(sym, x)
    assert nbits == 64 + 22 + 100
    got, esc = O.sz_stream_decode(data, nbits, 100)
    assert np.array_equal(got, sym) and esc.size == 0
    with pytest.raises(O.OracleError):
        O.sz_stream_decode(data, nbits - 1, 100)
    with pytest.raises(O.OracleError):
        O.sz_stream_decode(data + b"\x00", nbits + 8, 100)


def _zfp_stream_decode(data, nbits, nblocks, d, minexp):
    """Reads a fixed-accuracy ZFP stream back, written here from the stream's
    description: per block a flag, emax + 127 in 8 bits, then per plane from
    31 down to kmin = 32 - P (P = clamp(emax - minexp + 2(d+1), 0, 32)) the
    verbatim bits of the coefficients already significant and the group
    tests: a 1 means a one follows among the rest, found by scanning bits
    (the last coefficient's one implied).  Returns per block (emax or None,
    the coded planes of the negabinary coefficients)."""
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8))[:nbits]
    nb = 4 ** d
    pos = 0

    def rd(k=1):
        nonlocal pos
        v = 0
        for _ in range(k):
            v = (v << 1) | int(bits[pos])
            pos += 1
        return v

    out = []
    for _ in range(nblocks):
        if rd() == 0:
            out.append((None, [0] * nb))
            continue
        emax = rd(8) - 127
        kmin = 32 - min(32, max(0, emax - minexp + 2 * (d + 1)))
        u = [0] * nb
        n = 0
        for k in range(31, kmin - 1, -1):
            for j in range(n):
                u[j] |= rd() << k
            p = n
            while p < nb:
                if not rd():
                    break
                while p < nb - 1:
                    if rd():
                        break
                    p += 1
                u[p] |= 1 << k
                p += 1
                n = p
        out.append((emax, u))
    assert pos == nbits  # nothing left over
    return out


@pytest.mark.parametrize("shape,eb", [((37,), 1e-3), ((13, 18), 1e-4), ((9, 10, 11), 1e-2),
                                      ((8, 8, 8), 1e-6)])
def test_zfp_stream_carries_the_coded_planes(shape, eb):
    """The ZFP truth's bit count is the length of an embedded stream from
    which a decoder written from the description recovers every block's
    exponent and exactly the coded bit planes of its coefficients (all
    lower planes zero), block after block to the last bit."""
    x = (synth.grf_np(shape, -3.0, seed=len(shape) * 31) * 25.0).astype(np.float32)
    x.ravel()[::7] = 0.0
    p = O.params(eb=eb, r_sp=1.0)
    r = O.select(x, p)
    t = O.ground_truth(x, p)
    data, nbits = O.zfp_stream(x, r["eb_abs"])
    assert nbits == t["zfp_bits_gt"]
    zb = O.zfp_blocks(x, r["eb_abs"], want_coeffs=True)
    d = x.ndim
    minexp = math.frexp(r["eb_abs"])[1] - 1  # floor(log2 eb_abs), exactly
    dec = _zfp_stream_decode(data, nbits, len(zb["emax"]), d, minexp)
    for b, (emax, u) in enumerate(dec):
        if emax is None:
            assert zb["prec"][b] == 0
            continue
        assert emax == zb["emax"][b]
        keep = (0xFFFFFFFF << (32 - int(zb["prec"][b]))) & 0xFFFFFFFF
        assert u == [int(c) & keep for c in zb["coeffs"][b]], b


@pytest.mark.parametrize("shape,eb", [((37,), 1e-3), ((13, 18), 1e-4), ((9, 10, 11), 1e-2),
                                      ((20, 24, 28), 1e-5)])
def test_zfp_stream_rebuilds_the_field_within_the_bound(shape, eb):
    """The field read back from the ZFP stream alone is within eb_abs of the
    original at every point, and its squared and largest errors are those
    the ZFP ground truth reports."""
    x = (synth.grf_np(shape, -3.0, seed=len(shape) * 17) * 25.0).astype(np.float32)
    p = O.params(eb=eb, r_sp=1.0)
    r = O.select(x, p)
    t = O.ground_truth(x, p)
    data, nbits = O.zfp_stream(x, r["eb_abs"])
    rec = O.zfp_stream_decode(data, nbits, x.shape, r["eb_abs"])
    e = np.abs(x.astype(np.float64) - rec.astype(np.float64))
    assert e.max() <= r["eb_abs"]
    assert float(e.max()) == pytest.approx(t["maxerr_zfp"], rel=2.0 ** -23)
    assert float((e * e).sum()) == pytest.approx(t["sse_zfp"], rel=1e-12)
    with pytest.raises(O.OracleError):
        O.zfp_stream_decode(data, nbits - 1, x.shape, r["eb_abs"])
