"""Planted mutations: the definition pins must fail on a broken oracle.

Each case copies the oracle's C source to a temporary folder, plants one
plausible mistake (a natural logarithm for log2, a wrong total, a bin of
twice or half the width, a flipped sign, a wrong stencil neighbour), builds
it with the oracle's own flags and runs the pins of oracle_checks.py against
that build.  Every mutant must make at least one of its pins fail; the real
oracle passes them all (test_oracle_definitions.py).  Nothing here touches
the product path: the mutants are CPU builds of the checker.
"""
import contextlib
import os
import subprocess

import numpy as np
import pytest

import oracle_checks as C
import synth

O = pytest.importorskip("oracle")
from oracle import build as OB  # noqa: E402

# (source text, replacement) pairs per mutant, and the pins that must catch it
MUTANTS = {
    "entropy_natural_log": (
        [("H -= p * log2(p);", "H -= p * log(p);")], ["entropy"]),
    "entropy_wrong_total": (
        [("double p = (double)h[s] / (double)ns;",
          "double p = (double)h[s] / (double)(ns + 1);")], ["entropy"]),
    "estimator_twice_the_bin": (
        [("float q = rintf(r * inv);", "float q = rintf(r * inv * 0.5f);")], ["estimator"]),
    "estimator_sign_flip": (
        [("float q = rintf(r * inv);", "float q = rintf(-r * inv);")], ["estimator"]),
    "estimator_wrong_neighbour_2d": (
        [("int64_t e[2] = {idx[0] - 1, idx[1] - 1};", "int64_t e[2] = {idx[0] - 1, idx[1]};")],
        ["estimator"]),
    "estimator_wrong_neighbour_3d": (
        [("int64_t e[3] = {k, idx[1] - 1, idx[2] - 1};", "int64_t e[3] = {k, idx[1] - 1, idx[2]};")],
        ["estimator"]),
    "prequantiser_twice_the_bin": (
        [("Q[i] = (int32_t)rintf(f.x[i] * qz.inv);",
          "Q[i] = (int32_t)rintf(f.x[i] * qz.inv * 0.5f);")], ["truth"]),
    "prequantiser_sign_flip": (
        [("Q[i] = (int32_t)rintf(f.x[i] * qz.inv);", "Q[i] = (int32_t)rintf(-f.x[i] * qz.inv);")],
        ["truth"]),
    "prequantiser_half_bin_kept_in_bound": (
        # a bin of delta/2 used consistently: every error stays within delta/2
        [("Q[i] = (int32_t)rintf(f.x[i] * qz.inv);",
          "Q[i] = (int32_t)rintf(f.x[i] * qz.inv * 2.0f);"),
         ("float xh = (float)Q[i] * qz.w;", "float xh = (float)Q[i] * (qz.w * 0.5f);")],
        ["truth"]),
    "log_code_sign_flip": (
        [("return r < 0.0f ? -lo : lo;", "return r < 0.0f ? lo : -lo;")], ["log"]),
    "log_width_one_bin_down": (
        [("double w = k == 0 ? 2.0 * A[1] : A[k + 1] - A[k];",
          "double w = k == 0 ? 2.0 * A[1] : A[k] - A[k - 1];")], ["log"]),
    "log_edge_off_by_one_power": (
        [("for (int k = 1; k <= n; k++) A[k] = log_edge(u, b, k);",
          "for (int k = 1; k <= n; k++) A[k] = log_edge(u, b, k + 1);")], ["log"]),
    "truth_residual_sign": (
        [("r += odd ? -q_at(f, Q, j) : q_at(f, Q, j);", "r += odd ? q_at(f, Q, j) : -q_at(f, Q, j);")],
        ["truth"]),
}


def _fields():
    return [
        (synth.grf_np((1001,), -2.0, 401) * 25 + 100).astype(np.float32),
        (synth.grf_np((41, 37), -3.0, 402) * 25 + 100).astype(np.float32),
        (synth.grf_np((11, 13, 15), -3.0, 403) * 25 + 100).astype(np.float32),
    ]


def _run_pin(kind):
    if kind == "log":
        C.check_log_bins_and_mse(O)
        return
    if kind == "entropy":
        C.check_entropy_equal_bins(O)
        C.check_entropy_unequal_bins(O)
        return
    for x in _fields():
        vr = float(x.max()) - float(x.min())
        for rel in (1e-2, 1e-4):
            if kind == "estimator":
                C.estimator_disagreements(O, x, rel * vr * 1.0137)
            else:
                C.truth_disagreements(O, x, rel * vr * 0.9871)


@contextlib.contextmanager
def _oracle_build(lib_path):
    saved = O._lib
    O._lib = O.load(lib_path)
    try:
        yield
    finally:
        O._lib = saved


def _build_mutant(tmp_path, edits):
    with open(OB.SRC) as f:
        src = f.read()
    for old, new in edits:
        assert src.count(old) == 1, ("mutation site not unique", old)
        src = src.replace(old, new)
    cdir = tmp_path / "src"
    cdir.mkdir()
    (cdir / "rdo.c").write_text(src)
    with open(OB.HDR) as f:
        (cdir / "rdo.h").write_text(f.read())
    lib = str(tmp_path / "libmutant.so")
    subprocess.run(["gcc", *OB.CFLAGS, "-o", lib, str(cdir / "rdo.c"), "-lm"], check=True,
                   capture_output=True)
    return lib


def test_unmutated_copy_passes_every_pin(tmp_path):
    """The harness itself: a copy built the same way with no edit passes."""
    lib = _build_mutant(tmp_path, [])
    with _oracle_build(lib):
        for kind in ("entropy", "estimator", "truth", "log"):
            _run_pin(kind)


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    edits, kinds = MUTANTS[name]
    lib = _build_mutant(tmp_path, edits)
    caught = []
    with _oracle_build(lib):
        for kind in kinds:
            try:
                _run_pin(kind)
            except AssertionError:
                caught.append(kind)
    assert caught, f"mutant {name} passed every pin"
    os.remove(lib)
