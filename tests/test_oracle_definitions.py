"""Pins of the oracle's SZ quantisers and entropy against their plain
definitions (the checks live in oracle_checks.py, which the planted-mutation
tests reuse).

- The entropy (Eq. entropy, Eq. bitrate-sz) of histograms known in advance:
  exactly k bits for equal counts over 2^k codes, and an exactly summed
  reference on an unequal histogram.
- Every estimator code and every prequantised code against the float64
  definition floor(v / delta + 0.5) on seeded fields at several bin widths:
  the float32 decisions may differ only within their rounding error of a
  bin edge, by one bin; the number of such points is reported.
"""
import numpy as np
import pytest

import oracle_checks as C
import synth

O = pytest.importorskip("oracle")


def test_entropy_of_known_equal_histograms():
    C.check_entropy_equal_bins(O)


def test_entropy_of_known_unequal_histogram():
    C.check_entropy_unequal_bins(O)


def _fields():
    return {
        "1d": (synth.grf_np((4001,), -2.0, 301) * 25 + 100).astype(np.float32),
        "2d": (synth.grf_np((97, 83), -3.0, 302) * 25 + 100).astype(np.float32),
        "3d": (synth.grf_np((23, 29, 31), -3.0, 303) * 25 + 100).astype(np.float32),
        "3d_fronts": synth.config2_field(seed=304, shape=(20, 36, 40)),
    }


FIELDS = _fields()


def _few(out):
    """Where float32 resolves the bins (few points near an edge), at most one
    point in a thousand differs.  At eb_rel 1e-6 the bin nears the float
    spacing of the values, most points lie within rounding of an edge, and
    the check reduces to: differences of one bin, only at those points."""
    if out["near_edge"] * 10 < out["points"]:
        assert out["differ"] <= max(2, out["points"] // 1000), out


@pytest.mark.parametrize("name", list(FIELDS))
@pytest.mark.parametrize("rel", [1e-2, 1e-4, 1e-6])
def test_estimator_codes_follow_the_definition(name, rel):
    x = FIELDS[name]
    vr = float(x.max()) - float(x.min())
    # a bin width that is not a power of two times a short fraction
    delta = rel * vr * 1.0137
    out = C.estimator_disagreements(O, x, delta)
    print(f"estimator {name} rel={rel}: {out}")
    _few(out)


@pytest.mark.parametrize("name", list(FIELDS))
@pytest.mark.parametrize("rel", [1e-2, 1e-4, 1e-6])
def test_prequantised_codes_follow_the_definition(name, rel):
    x = FIELDS[name]
    vr = float(x.max()) - float(x.min())
    delta = rel * vr * 0.9871
    out = C.truth_disagreements(O, x, delta)
    print(f"truth {name} rel={rel}: {out}")
    _few(out)


def test_estimator_codes_with_escapes():
    """A small radius: codes at or beyond it escape (symbol 0), exactly where
    the definition's |q| >= R (up to a code on a bin edge)."""
    x = FIELDS["2d"]
    vr = float(x.max()) - float(x.min())
    out = C.estimator_disagreements(O, x, 1e-3 * vr, radius=16)
    assert out["escapes"] > 0
