"""ctypes wrapper of the CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow statement of the
online SZ-vs-ZFP rate-distortion estimation of Tao et al. (arXiv 1806.08901,
Algorithm 1 and Sections "Estimation Based on Static Quantization" and
"Estimation Based on Dynamic Quantization") and of the full-field ground truth
that judges it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
imports nothing from the CUDA package and the CUDA package imports nothing
from it.

Every function takes numpy arrays on the host and returns plain dicts.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

EB_REL, EB_ABS = 0, 1
EC_PAPER, EC_ALL = 0, 1
SEL_PAPER, SEL_HUFFMAN = 0, 1
F_CONSTANT, F_DELTA_CLAMPED, F_MSE_ZERO, F_TIE_BAND, F_PARTIAL_BLOCKS = 1, 2, 4, 8, 16
OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_RANGE = 0, -1, -2, -7
NSYM = 65536


class Params(C.Structure):
    _fields_ = [
        ("eb", C.c_double),
        ("eb_mode", C.c_int32),
        ("ec_mode", C.c_int32),
        ("r_sp", C.c_double),
        ("quant_radius", C.c_int32),
        ("sel_rule", C.c_int32),
        ("sz_offset", C.c_double),
    ]


class Result(C.Structure):
    _fields_ = [
        ("vmin", C.c_float),
        ("vmax", C.c_float),
        ("vr", C.c_double),
        ("eb_abs", C.c_double),
        ("r_sp_eff", C.c_double),
        ("strides", C.c_int32 * 3),
        ("minexp", C.c_int32),
        ("n_blocks", C.c_uint64),
        ("n_sampled_blocks", C.c_uint64),
        ("br_zfp", C.c_double),
        ("psnr_zfp", C.c_double),
        ("mse_sp", C.c_double),
        ("zfp_s2", C.c_uint64),
        ("zfp_npoints", C.c_uint64),
        ("zfp_ncoeff", C.c_uint64),
        ("delta", C.c_double),
        ("br_sz", C.c_double),
        ("br_sz_huff", C.c_double),
        ("psnr_sz", C.c_double),
        ("entropy", C.c_double),
        ("sz_ns", C.c_uint64),
        ("sz_huff_bits", C.c_uint64),
        ("sz_nesc", C.c_uint64),
        ("sz_nsym", C.c_uint32),
        ("selection", C.c_int32),
        ("flags", C.c_uint32),
    ]


class Truth(C.Structure):
    _fields_ = [
        ("eb_sz", C.c_double),
        ("delta", C.c_double),
        ("br_sz_gt", C.c_double),
        ("psnr_sz_gt", C.c_double),
        ("sse_sz", C.c_double),
        ("maxerr_sz", C.c_double),
        ("sz_bits_gt", C.c_uint64),
        ("sz_huff_gt", C.c_uint64),
        ("sz_nesc_gt", C.c_uint64),
        ("sz_nsym_gt", C.c_uint32),
        ("br_zfp_gt", C.c_double),
        ("psnr_zfp_gt", C.c_double),
        ("sse_zfp", C.c_double),
        ("maxerr_zfp", C.c_double),
        ("zfp_bits_gt", C.c_uint64),
        ("best_gt", C.c_int32),
        ("flags", C.c_uint32),
    ]


class LogResult(C.Structure):
    _fields_ = [
        ("vr", C.c_double),
        ("eb_abs", C.c_double),
        ("unit", C.c_double),
        ("max_abs", C.c_double),
        ("base", C.c_double),
        ("entropy", C.c_double),
        ("br_log", C.c_double),
        ("br_log_huff", C.c_double),
        ("mse_log", C.c_double),
        ("psnr_log", C.c_double),
        ("ns", C.c_uint64),
        ("huff_bits", C.c_uint64),
        ("nsym", C.c_uint32),
        ("flags", C.c_uint32),
    ]


class BlockOut(C.Structure):
    _fields_ = [
        ("emax", C.c_int32),
        ("prec", C.c_int32),
        ("kmin", C.c_int32),
        ("all_zero", C.c_int32),
        ("coeff_int", C.c_int32 * 64),
        ("coeff_nb", C.c_uint32 * 64),
        ("bits_emitter", C.c_uint64),
        ("bits_closed", C.c_uint64),
        ("s2_block", C.c_int64),
        ("nsb", C.c_int32 * 64),
        ("d", C.c_int64 * 64),
        ("recon", C.c_float * 64),
    ]


_lib = None


def load(path: str):
    """Open a build of the oracle at `path` and declare its signatures."""
    L = C.CDLL(path)
    P = C.POINTER
    f32p, i64p, i32p = P(C.c_float), P(C.c_int64), P(C.c_int32)
    u32p, u64p = P(C.c_uint32), P(C.c_uint64)
    sig = {
        "rdo_select": [f32p, C.c_int, i64p, P(Params), P(Result), u32p],
        "rdo_ground_truth": [f32p, C.c_int, i64p, P(Params), C.c_double, P(Truth), u32p],
        "rdo_estimate_sz": [f32p, C.c_int, i64p, P(Params), C.c_double, P(Result), u32p],
        "rdo_estimate_sz_log": [f32p, C.c_int, i64p, P(Params), P(LogResult), u32p,
                                P(C.c_double)],
        "rdo_zfp_blocks": [f32p, C.c_int, i64p, C.c_double, i32p, i32p, u64p, u32p],
        "rdo_sz_symbols": [f32p, C.c_int, i64p, C.c_double, C.c_int32, i32p, i32p, i32p, f32p],
        "rdo_zfp_block": [f32p, C.c_int, C.c_int32, C.c_int32, P(BlockOut)],
        "rdo_huffman_cost": [u64p, C.c_int64, u64p],
        "rdo_sequency": [C.c_int, i32p],
        "rdo_ec_positions": [C.c_int, C.c_int32, i32p, i32p],
        "rdo_sampling": [C.c_int, i64p, C.c_double, i32p, u64p, u64p],
        "rdo_mse_numerator": [i32p, i64p, C.c_int64, P(C.c_double)],
        "rdo_classic_sz": [f32p, C.c_int, i64p, P(Params), C.c_double, P(Truth), u32p, i32p,
                           f32p],
        "rdo_sz_stream_encode": [i32p, f32p, C.c_int64, P(C.c_uint8), C.c_uint64, u64p],
        "rdo_sz_stream_decode": [P(C.c_uint8), C.c_uint64, C.c_int64, i32p, u32p, C.c_uint64,
                                 u64p],
        "rdo_zfp_stream_encode": [f32p, C.c_int, i64p, C.c_double, P(C.c_uint8), C.c_uint64,
                                  u64p],
        "rdo_zfp_stream_decode": [P(C.c_uint8), C.c_uint64, C.c_int, i64p, C.c_double, f32p],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.rdo_fwd_lift.argtypes = [i32p]
    L.rdo_fwd_lift.restype = None
    L.rdo_inv_lift.argtypes = [i32p]
    L.rdo_inv_lift.restype = None
    L.rdo_int2nb.argtypes = [C.c_int32]
    L.rdo_int2nb.restype = C.c_uint32
    L.rdo_nb2int.argtypes = [C.c_uint32]
    L.rdo_nb2int.restype = C.c_int32
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _field(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim < 1 or x.ndim > 3:
        raise ValueError("fields are 1-, 2- or 3-dimensional")
    shape = np.array(x.shape, dtype=np.int64)
    return x, shape


def params(eb=1e-4, eb_mode=EB_REL, ec_mode=EC_PAPER, r_sp=0.05,
           quant_radius=32768, sel_rule=SEL_PAPER, sz_offset=0.5) -> Params:
    return Params(eb, eb_mode, ec_mode, r_sp, quant_radius, sel_rule, sz_offset)


def _todict(s: C.Structure) -> dict:
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        if isinstance(v, C.Array):
            v = list(v)
        out[name] = v
    return out


def select(x: np.ndarray, p: Params, want_hist: bool = False):
    x, shape = _field(x)
    r = Result()
    h = np.zeros(NSYM, dtype=np.uint32) if want_hist else None
    rc = lib().rdo_select(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                          C.byref(p), C.byref(r),
                          _ptr(h, C.c_uint32) if h is not None else None)
    if rc:
        raise OracleError(rc, "rdo_select")
    d = _todict(r)
    if want_hist:
        d["hist"] = h
    return d


def estimate_sz(x: np.ndarray, p: Params, delta: float = 0.0, want_hist: bool = False):
    x, shape = _field(x)
    r = Result()
    h = np.zeros(NSYM, dtype=np.uint32) if want_hist else None
    rc = lib().rdo_estimate_sz(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                               C.byref(p), float(delta), C.byref(r),
                               _ptr(h, C.c_uint32) if h is not None else None)
    if rc:
        raise OracleError(rc, "rdo_estimate_sz")
    d = _todict(r)
    if want_hist:
        d["hist"] = h
    return d


def estimate_sz_log(x: np.ndarray, p: Params, want_hist: bool = False, want_edges: bool = False):
    """Log-scale quantisation estimate; edges: A[1..n] (n = quant_radius)."""
    x, shape = _field(x)
    r = LogResult()
    h = np.zeros(NSYM, dtype=np.uint32) if want_hist else None
    e = np.zeros(p.quant_radius, dtype=np.float64) if want_edges else None
    rc = lib().rdo_estimate_sz_log(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                                   C.byref(p), C.byref(r),
                                   _ptr(h, C.c_uint32) if h is not None else None,
                                   _ptr(e, C.c_double) if e is not None else None)
    if rc:
        raise OracleError(rc, "rdo_estimate_sz_log")
    out = _todict(r)
    if want_hist:
        out["hist"] = h
    if want_edges:
        out["edges"] = e
    return out


def ground_truth(x: np.ndarray, p: Params, eb_sz: float = 0.0, want_hist: bool = False):
    x, shape = _field(x)
    t = Truth()
    h = np.zeros(NSYM, dtype=np.uint32) if want_hist else None
    rc = lib().rdo_ground_truth(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                                C.byref(p), float(eb_sz), C.byref(t),
                                _ptr(h, C.c_uint32) if h is not None else None)
    if rc:
        raise OracleError(rc, "rdo_ground_truth")
    d = _todict(t)
    if want_hist:
        d["hist"] = h
    return d


def classic_sz(x: np.ndarray, p: Params, eb_sz: float, want_hist: bool = False,
               want_recon: bool = False, want_sym: bool = False):
    """Classic SZ at the absolute bound eb_sz (Section "Prediction-Based
    Transformation": prediction from the reconstructed neighbours, point by
    point in storage order).  Returns the SZ fields of the truth record, and
    the histogram and reconstruction when asked."""
    x, shape = _field(x)
    t = Truth()
    h = np.zeros(NSYM, dtype=np.uint32) if want_hist else None
    r = np.zeros(x.shape, dtype=np.float32) if want_recon else None
    sy = np.zeros(x.shape, dtype=np.int32) if want_sym else None
    rc = lib().rdo_classic_sz(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64), C.byref(p),
                              float(eb_sz), C.byref(t),
                              _ptr(h, C.c_uint32) if h is not None else None,
                              _ptr(sy, C.c_int32) if sy is not None else None,
                              _ptr(r, C.c_float) if r is not None else None)
    if rc:
        raise OracleError(rc, "rdo_classic_sz")
    d = _todict(t)
    if want_hist:
        d["hist"] = h
    if want_recon:
        d["recon"] = r
    if want_sym:
        d["sym"] = sy
    return d


def rd_curve(x: np.ndarray, p: Params, ebs) -> list:
    """Rate-distortion points over the bounds ebs (evaluation section,
    "Analysis of Adaptability between Selection Methods Based on Fixed-PSNR
    vs. Fixed-Maximum-Error", Fig. f9, and the "optimum bar" of Fig. f5).  At
    each bound: Algorithm 1 (select) and its ground truth at the matched PSNR
    (SZ at delta/2; best_gt is the optimum choice); and the selection based on
    error bound that the paper compares against, both compressors at the same
    maximum error eb_abs: SZ with bin 2 eb_abs (estimate_sz with delta 0)
    against ZFP at eb_abs, SZ iff its bit-rate is lower, from the estimates
    and from the ground truth at eb_sz = eb_abs."""
    out = []
    for eb in ebs:
        q = Params(float(eb), p.eb_mode, p.ec_mode, p.r_sp, p.quant_radius, p.sel_rule,
                   p.sz_offset)
        est = select(x, q)
        truth = ground_truth(x, q)
        est_eb = estimate_sz(x, q, delta=0.0)
        truth_eb = ground_truth(x, q, eb_sz=est["eb_abs"]) if est["eb_abs"] > 0.0 else None
        br = est_eb["br_sz_huff"] if p.sel_rule == SEL_HUFFMAN else est_eb["br_sz"]
        out.append(dict(eb=float(eb), est=est, truth=truth, est_eb=est_eb, truth_eb=truth_eb,
                        selection_eb=0 if br < est["br_zfp"] else 1,
                        best_eb_gt=truth_eb["best_gt"] if truth_eb is not None else 0))
    return out


def zfp_blocks(x: np.ndarray, eb_abs: float, want_coeffs: bool = False):
    x, shape = _field(x)
    nblk = int(np.prod([(n + 3) // 4 for n in x.shape]))
    nb = 4 ** x.ndim
    emax = np.zeros(nblk, np.int32)
    prec = np.zeros(nblk, np.int32)
    bits = np.zeros(nblk, np.uint64)
    coeffs = np.zeros(nblk * nb, np.uint32) if want_coeffs else None
    rc = lib().rdo_zfp_blocks(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                              float(eb_abs), _ptr(emax, C.c_int32), _ptr(prec, C.c_int32),
                              _ptr(bits, C.c_uint64),
                              _ptr(coeffs, C.c_uint32) if coeffs is not None else None)
    if rc:
        raise OracleError(rc, "rdo_zfp_blocks")
    out = {"emax": emax, "prec": prec, "bits": bits}
    if want_coeffs:
        out["coeffs"] = coeffs.reshape(nblk, nb)
    return out


def sz_symbols(x: np.ndarray, delta: float, quant_radius: int = 32768, strides=None):
    x, shape = _field(x)
    n = x.size
    est = np.full(n, -1, np.int32)
    gt = np.zeros(n, np.int32)
    rec = np.zeros(n, np.float32)
    st = None
    if strides is not None:
        st = np.array(list(strides) + [1] * (3 - len(strides)), dtype=np.int32)
    rc = lib().rdo_sz_symbols(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                              float(delta), int(quant_radius),
                              _ptr(st, C.c_int32) if st is not None else None,
                              _ptr(est, C.c_int32), _ptr(gt, C.c_int32), _ptr(rec, C.c_float))
    if rc:
        raise OracleError(rc, "rdo_sz_symbols")
    return {"est": est.reshape(x.shape), "gt": gt.reshape(x.shape), "recon": rec.reshape(x.shape)}


def sz_stream(sym: np.ndarray, x: np.ndarray):
    """The SZ stream of the symbols sym (0 = escape: x stored as its 32-bit
    pattern), as the ground-truth bit counts cost it.  Returns (bytes, nbits)."""
    sym = np.ascontiguousarray(sym, dtype=np.int32).ravel()
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    if sym.size != x.size:
        raise ValueError("one value per symbol")
    nbits = C.c_uint64(0)
    rc = lib().rdo_sz_stream_encode(_ptr(sym, C.c_int32), _ptr(x, C.c_float), sym.size, None, 0,
                                    C.byref(nbits))
    if rc:
        raise OracleError(rc, "rdo_sz_stream_encode")
    buf = np.zeros((nbits.value + 7) // 8, dtype=np.uint8)
    rc = lib().rdo_sz_stream_encode(_ptr(sym, C.c_int32), _ptr(x, C.c_float), sym.size,
                                    _ptr(buf, C.c_uint8), buf.size, C.byref(nbits))
    if rc:
        raise OracleError(rc, "rdo_sz_stream_encode")
    return buf.tobytes(), nbits.value


def zfp_stream(x: np.ndarray, eb_abs: float):
    """The fixed-accuracy ZFP stream of the field at eb_abs (the stream the
    ZFP ground-truth bit count costs).  Returns (bytes, nbits)."""
    x, shape = _field(x)
    nbits = C.c_uint64(0)
    rc = lib().rdo_zfp_stream_encode(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                                     float(eb_abs), None, 0, C.byref(nbits))
    if rc:
        raise OracleError(rc, "rdo_zfp_stream_encode")
    buf = np.zeros((nbits.value + 7) // 8, dtype=np.uint8)
    rc = lib().rdo_zfp_stream_encode(_ptr(x, C.c_float), x.ndim, _ptr(shape, C.c_int64),
                                     float(eb_abs), _ptr(buf, C.c_uint8), buf.size, C.byref(nbits))
    if rc:
        raise OracleError(rc, "rdo_zfp_stream_encode")
    return buf.tobytes(), nbits.value


def zfp_stream_decode(data: bytes, nbits: int, shape, eb_abs: float) -> np.ndarray:
    """The field a fixed-accuracy ZFP stream encodes."""
    buf = np.frombuffer(data, dtype=np.uint8).copy()
    shape = tuple(int(s) for s in shape)
    sh = np.array(list(shape) + [1] * (3 - len(shape)), dtype=np.int64)
    rec = np.zeros(shape, np.float32)
    rc = lib().rdo_zfp_stream_decode(_ptr(buf, C.c_uint8), int(nbits), len(shape),
                                     _ptr(sh, C.c_int64), float(eb_abs), _ptr(rec, C.c_float))
    if rc:
        raise OracleError(rc, "rdo_zfp_stream_decode")
    return rec


def sz_stream_decode(data: bytes, nbits: int, n: int):
    """Symbols and escaped values (float32) read back from an SZ stream."""
    buf = np.frombuffer(data, dtype=np.uint8).copy()
    sym = np.zeros(n, np.int32)
    esc = np.zeros(max(n, 1), np.uint32)
    ne = C.c_uint64(0)
    rc = lib().rdo_sz_stream_decode(_ptr(buf, C.c_uint8), int(nbits), int(n), _ptr(sym, C.c_int32),
                                    _ptr(esc, C.c_uint32), esc.size, C.byref(ne))
    if rc:
        raise OracleError(rc, "rdo_sz_stream_decode")
    return sym, esc[: ne.value].view(np.float32)


def zfp_block(v: np.ndarray, ndim: int, minexp: int, ec_mode: int = EC_PAPER) -> dict:
    v = np.ascontiguousarray(v, dtype=np.float32).ravel()
    if v.size != 4 ** ndim:
        raise ValueError("a block holds 4^d values")
    o = BlockOut()
    rc = lib().rdo_zfp_block(_ptr(v, C.c_float), ndim, int(minexp), int(ec_mode), C.byref(o))
    if rc:
        raise OracleError(rc, "rdo_zfp_block")
    d = _todict(o)
    nb = 4 ** ndim
    for k in ("coeff_int", "coeff_nb", "nsb", "d", "recon"):
        d[k] = d[k][:nb]
    return d


def huffman_cost(counts) -> int:
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
    out = C.c_uint64()
    rc = lib().rdo_huffman_cost(_ptr(c, C.c_uint64), c.size, C.byref(out))
    if rc:
        raise OracleError(rc, "rdo_huffman_cost")
    return int(out.value)


def fwd_lift(v4) -> list:
    a = np.ascontiguousarray(np.asarray(v4, dtype=np.int32))
    lib().rdo_fwd_lift(_ptr(a, C.c_int32))
    return [int(t) for t in a]


def inv_lift(v4) -> list:
    a = np.ascontiguousarray(np.asarray(v4, dtype=np.int32))
    lib().rdo_inv_lift(_ptr(a, C.c_int32))
    return [int(t) for t in a]


def int2nb(i: int) -> int:
    return int(lib().rdo_int2nb(int(i)))


def nb2int(u: int) -> int:
    return int(lib().rdo_nb2int(int(u)))


def sequency(ndim: int) -> list:
    perm = np.zeros(64, np.int32)
    rc = lib().rdo_sequency(ndim, _ptr(perm, C.c_int32))
    if rc:
        raise OracleError(rc, "rdo_sequency")
    return [int(t) for t in perm[: 4 ** ndim]]


def ec_positions(ndim: int, ec_mode: int = EC_PAPER) -> list:
    pos = np.zeros(64, np.int32)
    m = C.c_int32()
    rc = lib().rdo_ec_positions(ndim, ec_mode, _ptr(pos, C.c_int32), C.byref(m))
    if rc:
        raise OracleError(rc, "rdo_ec_positions")
    return [int(t) for t in pos[: m.value]]


def sampling(shape, r_sp: float):
    sh = np.array(shape, dtype=np.int64)
    st = np.zeros(3, np.int32)
    nsb = C.c_uint64()
    npts = C.c_uint64()
    rc = lib().rdo_sampling(len(shape), _ptr(sh, C.c_int64), float(r_sp),
                            _ptr(st, C.c_int32), C.byref(nsb), C.byref(npts))
    if rc:
        raise OracleError(rc, "rdo_sampling")
    return [int(t) for t in st[: len(shape)]], int(nsb.value), int(npts.value)


def mse_numerator(emax, d) -> float:
    e = np.ascontiguousarray(np.asarray(emax, dtype=np.int32))
    dd = np.ascontiguousarray(np.asarray(d, dtype=np.int64))
    out = C.c_double()
    rc = lib().rdo_mse_numerator(_ptr(e, C.c_int32), _ptr(dd, C.c_int64), e.size, C.byref(out))
    if rc:
        raise OracleError(rc, "rdo_mse_numerator")
    return float(out.value)


def psnr(vr: float, mse: float) -> float:
    """Eq. (psnr-pdf): PSNR = 20 log10(VR) - 10 log10(MSE)."""
    if mse <= 0:
        return math.inf
    return 20.0 * math.log10(vr) - 10.0 * math.log10(mse)
