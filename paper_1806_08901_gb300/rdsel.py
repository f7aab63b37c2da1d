"""ctypes binding of ``librdsel.so`` (include/rdsel.h): argument marshalling
only.  Every step of the rate-distortion path runs in the library's CUDA
kernels; this module turns tensors into rd_field records, calls the C entry
point of the same name and turns the result records into dicts.

There is no fallback: if the library is missing or cannot load, every call
raises ``RdselUnavailable``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librdsel.so")

RD_OK = 0
RD_ERR_INVALID_ARG, RD_ERR_NONFINITE, RD_ERR_OOM = -1, -2, -3
RD_ERR_BUDGET, RD_ERR_CUDA, RD_ERR_TIMEOUT, RD_ERR_RANGE = -4, -5, -6, -7
RD_EB_REL, RD_EB_ABS = 0, 1
RD_EC_PAPER, RD_EC_ALL = 0, 1
RD_SEL_PAPER, RD_SEL_HUFFMAN = 0, 1
RD_LOC_DEVICE, RD_LOC_HOST = 0, 1
RD_F_CONSTANT, RD_F_DELTA_CLAMPED, RD_F_MSE_ZERO = 1, 2, 4
RD_F_TIE_BAND, RD_F_PARTIAL_BLOCKS = 8, 16
RD_NSYM = 65536


class RdselUnavailable(RuntimeError):
    pass


class RdselError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str = ""):
        super().__init__(f"{what}: {msg} (status {code})")
        self.code = code


class rd_field(C.Structure):
    _fields_ = [("data", C.c_void_p), ("ndim", C.c_int32), ("location", C.c_int32),
                ("shape", C.c_int64 * 3)]


class rd_params(C.Structure):
    _fields_ = [("eb", C.c_double), ("eb_mode", C.c_int32), ("ec_mode", C.c_int32),
                ("r_sp", C.c_double), ("quant_radius", C.c_int32), ("sel_rule", C.c_int32),
                ("sz_offset", C.c_double)]


class rd_result(C.Structure):
    _fields_ = [
        ("vmin", C.c_float), ("vmax", C.c_float), ("vr", C.c_double), ("eb_abs", C.c_double),
        ("r_sp_eff", C.c_double), ("strides", C.c_int32 * 3), ("minexp", C.c_int32),
        ("n_blocks", C.c_uint64), ("n_sampled_blocks", C.c_uint64),
        ("br_zfp", C.c_double), ("psnr_zfp", C.c_double), ("mse_sp", C.c_double),
        ("zfp_s2", C.c_uint64), ("zfp_npoints", C.c_uint64), ("zfp_ncoeff", C.c_uint64),
        ("delta", C.c_double), ("br_sz", C.c_double), ("br_sz_huff", C.c_double),
        ("psnr_sz", C.c_double), ("entropy", C.c_double),
        ("sz_ns", C.c_uint64), ("sz_huff_bits", C.c_uint64), ("sz_nesc", C.c_uint64),
        ("sz_nsym", C.c_uint32), ("selection", C.c_int32), ("flags", C.c_uint32),
    ]


class rd_truth(C.Structure):
    _fields_ = [
        ("eb_sz", C.c_double), ("delta", C.c_double),
        ("br_sz_gt", C.c_double), ("psnr_sz_gt", C.c_double), ("sse_sz", C.c_double),
        ("maxerr_sz", C.c_double),
        ("sz_bits_gt", C.c_uint64), ("sz_huff_gt", C.c_uint64), ("sz_nesc_gt", C.c_uint64),
        ("sz_nsym_gt", C.c_uint32),
        ("br_zfp_gt", C.c_double), ("psnr_zfp_gt", C.c_double), ("sse_zfp", C.c_double),
        ("maxerr_zfp", C.c_double), ("zfp_bits_gt", C.c_uint64),
        ("best_gt", C.c_int32), ("flags", C.c_uint32),
    ]


class rd_log_result(C.Structure):
    _fields_ = [("vr", C.c_double), ("eb_abs", C.c_double), ("unit", C.c_double),
                ("max_abs", C.c_double), ("base", C.c_double), ("entropy", C.c_double),
                ("br_log", C.c_double), ("br_log_huff", C.c_double), ("mse_log", C.c_double),
                ("psnr_log", C.c_double), ("ns", C.c_uint64), ("huff_bits", C.c_uint64),
                ("nsym", C.c_uint32), ("flags", C.c_uint32)]


class rd_rd_point(C.Structure):
    _fields_ = [("eb", C.c_double), ("est", rd_result), ("truth", rd_truth), ("est_eb", rd_result),
                ("truth_eb", rd_truth), ("selection_eb", C.c_int32), ("best_eb_gt", C.c_int32)]


class rd_batch_config(C.Structure):
    _fields_ = [("range_values", C.c_int64), ("zfp_blocks", C.c_int32), ("sz_blocks", C.c_int32),
                ("ctas", C.c_int32), ("tuned", C.c_int32)]


class rd_server_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("window", C.c_int32),
                ("pad", C.c_int32), ("hbm_budget", C.c_uint64)]


class rd_server_completion(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int32),
                ("resident_hit", C.c_int32), ("queue_ms", C.c_double), ("service_ms", C.c_double),
                ("latency_ms", C.c_double), ("result", rd_result)]


class rd_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("pending", C.c_uint64), ("resident_hits", C.c_uint64), ("evictions", C.c_uint64),
                ("resident_fields", C.c_uint64), ("resident_bytes", C.c_uint64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double)]


# Every symbol include/rdsel.h declares, with its ctypes signature.
_P = C.POINTER
_SIGNATURES = {
    "rd_context_create": (C.c_int32, [C.c_int32, C.c_size_t, _P(C.c_void_p)]),
    "rd_context_destroy": (C.c_int32, [C.c_void_p]),
    "rd_estimate_zfp": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), _P(rd_result), C.c_void_p]),
    "rd_estimate_sz_log": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), _P(rd_log_result),
                                       C.c_void_p]),
    "rd_estimate_sz": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_double,
                                   _P(rd_result), C.c_void_p]),
    "rd_select": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), _P(rd_result), C.c_void_p]),
    "rd_ground_truth": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_double,
                                    _P(rd_truth), C.c_void_p]),
    "rd_ground_truth_classic": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_double,
                                            _P(rd_truth), C.c_void_p, C.c_void_p]),
    "rd_sz_compress": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_double, C.c_void_p,
                                   C.c_uint64, _P(C.c_uint64), C.c_void_p]),
    "rd_zfp_compress": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_void_p, C.c_uint64,
                                    _P(C.c_uint64), C.c_void_p]),
    "rd_compress": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_void_p, C.c_uint64,
                                _P(C.c_uint64), _P(C.c_int32), _P(rd_result), C.c_void_p]),
    "rd_rd_curve": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), _P(C.c_double), C.c_int32,
                                _P(rd_rd_point), C.c_void_p]),
    "rd_evaluate": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), _P(rd_result),
                                _P(rd_truth), C.c_void_p]),
    "rd_select_static": (C.c_int32, [_P(rd_field), _P(rd_params), _P(rd_result), C.c_void_p]),
    "rd_select_batch": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_int32,
                                    _P(rd_result), _P(rd_truth), _P(C.c_int32), C.c_void_p]),
    "rd_batch_set_config": (C.c_int32, [C.c_void_p, _P(rd_batch_config)]),
    "rd_batch_get_config": (C.c_int32, [C.c_void_p, _P(rd_batch_config)]),
    "rd_server_create": (C.c_int32, [_P(rd_server_config), _P(C.c_void_p)]),
    "rd_server_submit": (C.c_int32, [C.c_void_p, _P(rd_field), _P(rd_params), C.c_uint64,
                                     C.c_uint64, _P(C.c_uint64)]),
    "rd_server_poll": (C.c_int32, [C.c_void_p, _P(rd_server_completion), C.c_int32, C.c_int32,
                                   _P(C.c_int32)]),
    "rd_server_get_stats": (C.c_int32, [C.c_void_p, _P(rd_server_stats)]),
    "rd_server_reset_stats": (C.c_int32, [C.c_void_p]),
    "rd_server_destroy": (C.c_int32, [C.c_void_p]),
    "rd_copy_histograms": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rd_zfp_blocks": (C.c_int32, [C.c_void_p, _P(rd_field), C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "rd_sz_symbols": (C.c_int32, [C.c_void_p, _P(rd_field), C.c_double, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rd_set_profiling": (C.c_int32, [C.c_void_p, C.c_int32]),
    "rd_reset_profile": (C.c_int32, [C.c_void_p]),
    "rd_kernel_stat": (C.c_int32, [C.c_void_p, C.c_int32, _P(C.c_char_p), _P(C.c_double),
                                   _P(C.c_int64)]),
    "rd_launch_count": (C.c_int64, [C.c_void_p]),
    "rd_status_string": (C.c_char_p, [C.c_int32]),
}

_lib = None


def lib():
    """Load librdsel.so (once).  Raises RdselUnavailable if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RdselUnavailable(
                f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        try:
            L = C.CDLL(LIB_PATH)
        except OSError as e:
            raise RdselUnavailable(f"cannot load {LIB_PATH}: {e}") from e
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list:
    return list(_SIGNATURES)


def status_string(code: int) -> str:
    return lib().rd_status_string(int(code)).decode()


def _check(rc: int, what: str):
    if rc != RD_OK:
        raise RdselError(rc, what, status_string(rc))


def params(eb=1e-4, eb_mode=RD_EB_REL, ec_mode=RD_EC_PAPER, r_sp=0.05, quant_radius=32768,
           sel_rule=RD_SEL_PAPER, sz_offset=0.5) -> rd_params:
    return rd_params(eb, eb_mode, ec_mode, r_sp, quant_radius, sel_rule, sz_offset)


def _todict(s: C.Structure) -> dict:
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        out[name] = list(v) if isinstance(v, C.Array) else v
    return out


def make_field(x) -> tuple:
    """rd_field for a float32 C-contiguous torch tensor (device or host) or
    numpy array (host).  Returns (rd_field, keepalive)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("fields are contiguous float32 tensors")
        loc = RD_LOC_DEVICE if x.is_cuda else RD_LOC_HOST
        ptr, shape, keep = x.data_ptr(), tuple(x.shape), x
    else:
        a = np.asarray(x)
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("fields are C-contiguous float32 arrays")
        loc, ptr, shape, keep = RD_LOC_HOST, a.ctypes.data, a.shape, a
    if not 1 <= len(shape) <= 3:
        raise ValueError("fields are 1-, 2- or 3-dimensional")
    sh = (C.c_int64 * 3)(*(list(shape) + [1] * (3 - len(shape))))
    return rd_field(ptr, len(shape), loc, sh), keep


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


# ---------------------------------------------------------------------------
# Entry points, named as in include/rdsel.h
# ---------------------------------------------------------------------------

def rd_context_create(device: int = 0, hbm_budget: int = 0):
    h = C.c_void_p()
    _check(lib().rd_context_create(int(device), int(hbm_budget), C.byref(h)), "rd_context_create")
    return h


def rd_context_destroy(ctx) -> None:
    _check(lib().rd_context_destroy(ctx), "rd_context_destroy")


def rd_estimate_zfp(ctx, field, prm: rd_params, stream=None) -> dict:
    f, keep = make_field(field)
    r = rd_result()
    _check(lib().rd_estimate_zfp(ctx, C.byref(f), C.byref(prm), C.byref(r), _stream(stream)),
           "rd_estimate_zfp")
    return _todict(r)


def rd_estimate_sz(ctx, field, prm: rd_params, delta: float = 0.0, stream=None) -> dict:
    f, keep = make_field(field)
    r = rd_result()
    _check(lib().rd_estimate_sz(ctx, C.byref(f), C.byref(prm), float(delta), C.byref(r),
                                _stream(stream)), "rd_estimate_sz")
    return _todict(r)


def rd_estimate_sz_log(ctx, field, prm: rd_params, stream=None) -> dict:
    """The log-scale quantisation estimate of one field."""
    f, keep = make_field(field)
    r = rd_log_result()
    _check(lib().rd_estimate_sz_log(ctx, C.byref(f), C.byref(prm), C.byref(r), _stream(stream)),
           "rd_estimate_sz_log")
    return _todict(r)


def rd_select(ctx, field, prm: rd_params, stream=None) -> dict:
    f, keep = make_field(field)
    r = rd_result()
    _check(lib().rd_select(ctx, C.byref(f), C.byref(prm), C.byref(r), _stream(stream)), "rd_select")
    return _todict(r)


def rd_select_static(field, prm: rd_params, stream=None) -> dict:
    """rd_select without a context, on the library's fixed scratch array (for
    callers that may not allocate): device fields only; calls on one device
    must not overlap."""
    f, keep = make_field(field)
    r = rd_result()
    _check(lib().rd_select_static(C.byref(f), C.byref(prm), C.byref(r), _stream(stream)),
           "rd_select_static")
    return _todict(r)


def rd_ground_truth(ctx, field, prm: rd_params, eb_sz: float = 0.0, stream=None) -> dict:
    f, keep = make_field(field)
    t = rd_truth()
    _check(lib().rd_ground_truth(ctx, C.byref(f), C.byref(prm), float(eb_sz), C.byref(t),
                                 _stream(stream)), "rd_ground_truth")
    return _todict(t)


def rd_ground_truth_classic(ctx, field, prm: rd_params, eb_sz: float, recon=None,
                            stream=None) -> dict:
    """Classic SZ truth at the absolute bound eb_sz; recon, when given, is a
    contiguous float32 device tensor of the field's size that receives the
    reconstruction."""
    f, keep = make_field(field)
    t = rd_truth()
    rp = None
    if recon is not None:
        import torch
        n = int(np.prod([f.shape[k] for k in range(f.ndim)]))
        if not (isinstance(recon, torch.Tensor) and recon.is_cuda and recon.dtype == torch.float32
                and recon.is_contiguous() and recon.numel() == n):
            raise ValueError("recon must be a contiguous float32 CUDA tensor of the field's size")
        rp = C.c_void_p(recon.data_ptr())
    _check(lib().rd_ground_truth_classic(ctx, C.byref(f), C.byref(prm), float(eb_sz), C.byref(t),
                                         rp, _stream(stream)), "rd_ground_truth_classic")
    return _todict(t)


def rd_sz_compress(ctx, field, prm: rd_params, eb_sz: float, out=None, stream=None) -> int:
    """The SZ stream of the prequantised ground truth at eb_sz (layout in
    include/rdsel_stream.h) into out, a uint8 CUDA tensor of at least
    8 * ceil(nbits / 64) bytes (8-byte aligned); out=None only sizes it.
    Returns the stream's length in bits."""
    f, keep = make_field(field)
    nbits = C.c_uint64(0)
    ptr, cap = None, 0
    if out is not None:
        import torch
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.uint8
                and out.is_contiguous()):
            raise ValueError("out must be a contiguous uint8 CUDA tensor")
        ptr, cap = C.c_void_p(out.data_ptr()), out.numel()
    _check(lib().rd_sz_compress(ctx, C.byref(f), C.byref(prm), float(eb_sz), ptr, cap,
                                C.byref(nbits), _stream(stream)), "rd_sz_compress")
    return nbits.value


def _stream_out(out):
    if out is None:
        return None, 0
    import torch
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.uint8
            and out.is_contiguous()):
        raise ValueError("out must be a contiguous uint8 CUDA tensor")
    return C.c_void_p(out.data_ptr()), out.numel()


def rd_zfp_compress(ctx, field, prm: rd_params, out=None, stream=None) -> int:
    """The ZFP fixed-accuracy stream at eb_abs (layout in
    include/rdsel_stream.h) into out, a uint8 CUDA tensor of at least
    8 * ceil(nbits / 64) bytes; out=None only sizes it.  Returns the
    stream's length in bits."""
    f, keep = make_field(field)
    nbits = C.c_uint64(0)
    ptr, cap = _stream_out(out)
    _check(lib().rd_zfp_compress(ctx, C.byref(f), C.byref(prm), ptr, cap, C.byref(nbits),
                                 _stream(stream)), "rd_zfp_compress")
    return nbits.value


def rd_compress(ctx, field, prm: rd_params, out=None, stream=None) -> dict:
    """Algorithm 1 to the end: the selection s_i and the selected
    compressor's stream C_i (into out when given).  Returns selection,
    nbits and the selection's record (est)."""
    f, keep = make_field(field)
    nbits = C.c_uint64(0)
    sel = C.c_int32(-1)
    est = rd_result()
    ptr, cap = _stream_out(out)
    _check(lib().rd_compress(ctx, C.byref(f), C.byref(prm), ptr, cap, C.byref(nbits), C.byref(sel),
                             C.byref(est), _stream(stream)), "rd_compress")
    return {"selection": sel.value, "nbits": nbits.value, "est": _todict(est)}


def rd_rd_curve(ctx, field, prm: rd_params, ebs, stream=None) -> list:
    """Rate-distortion points over the bounds ebs: one dict per bound with
    eb, est, truth, est_eb, truth_eb (dicts) and selection_eb, best_eb_gt."""
    f, keep = make_field(field)
    n = len(ebs)
    eb = (C.c_double * n)(*[float(e) for e in ebs])
    out = (rd_rd_point * n)()
    _check(lib().rd_rd_curve(ctx, C.byref(f), C.byref(prm), eb, n, out, _stream(stream)), "rd_rd_curve")
    res = []
    for pt in out:
        res.append({"eb": pt.eb, "est": _todict(pt.est), "truth": _todict(pt.truth),
                    "est_eb": _todict(pt.est_eb), "truth_eb": _todict(pt.truth_eb),
                    "selection_eb": pt.selection_eb, "best_eb_gt": pt.best_eb_gt})
    return res


def rd_evaluate(ctx, field, prm: rd_params, stream=None) -> tuple:
    f, keep = make_field(field)
    r, t = rd_result(), rd_truth()
    _check(lib().rd_evaluate(ctx, C.byref(f), C.byref(prm), C.byref(r), C.byref(t),
                             _stream(stream)), "rd_evaluate")
    return _todict(r), _todict(t)


def rd_select_batch(ctx, fields, prms, truth: bool = False, stream=None, check: bool = True):
    """Estimates (and, with truth=True, ground truths) of many device fields
    in one batched call.  prms: one rd_params for all fields or a list.
    Returns (results, truths or None, statuses); raises on a call-level
    error, and on a per-field error when check is true."""
    n = len(fields)
    if isinstance(prms, rd_params):
        prms = [prms] * n
    if len(prms) != n or n < 1:
        raise ValueError("one rd_params per field")
    fs = (rd_field * n)()
    keep = []
    for i, x in enumerate(fields):
        f, k = make_field(x)
        fs[i] = f
        keep.append(k)
    ps = (rd_params * n)(*prms)
    rs = (rd_result * n)()
    ts = (rd_truth * n)() if truth else None
    st = (C.c_int32 * n)()
    rc = lib().rd_select_batch(ctx, fs, ps, n, rs, ts, st, _stream(stream))
    statuses = list(st)
    if rc != RD_OK and (check or all(v == rc for v in statuses)):
        raise RdselError(rc, "rd_select_batch", status_string(rc))
    return ([_todict(r) for r in rs], [_todict(t) for t in ts] if truth else None, statuses)


class BatchCall:
    """A batch call marshalled once (fields, parameters and output arrays), to
    be issued repeatedly with run(); for timing loops that must not pay the
    per-call marshalling."""

    def __init__(self, ctx, fields, prms, truth: bool = False):
        n = len(fields)
        if isinstance(prms, rd_params):
            prms = [prms] * n
        self.ctx, self.n = ctx, n
        self.fs = (rd_field * n)()
        self.keep = []
        for i, x in enumerate(fields):
            f, k = make_field(x)
            self.fs[i] = f
            self.keep.append(k)
        self.ps = (rd_params * n)(*prms)
        self.rs = (rd_result * n)()
        self.ts = (rd_truth * n)() if truth else None
        self.st = (C.c_int32 * n)()

    def run(self, stream=None) -> int:
        return lib().rd_select_batch(self.ctx, self.fs, self.ps, self.n, self.rs, self.ts,
                                     self.st, _stream(stream))

    def results(self) -> list:
        return [_todict(r) for r in self.rs]


def rd_batch_set_config(ctx, cfg=None) -> None:
    """Force the work split of later batch calls (a dict of rd_batch_config
    fields, zeros = defaults), or None for the autotuner."""
    if cfg is None:
        _check(lib().rd_batch_set_config(ctx, None), "rd_batch_set_config")
        return
    c = rd_batch_config()
    for k, v in cfg.items():
        setattr(c, k, int(v))
    _check(lib().rd_batch_set_config(ctx, C.byref(c)), "rd_batch_set_config")


def rd_batch_get_config(ctx) -> dict:
    c = rd_batch_config()
    _check(lib().rd_batch_get_config(ctx, C.byref(c)), "rd_batch_get_config")
    return _todict(c)


def rd_copy_histograms(ctx) -> tuple:
    est = np.zeros(RD_NSYM, np.uint32)
    gt = np.zeros(RD_NSYM, np.uint32)
    _check(lib().rd_copy_histograms(ctx, _ptr(est), _ptr(gt)), "rd_copy_histograms")
    return est, gt


def rd_zfp_blocks(ctx, field, eb_abs: float, want_coeffs: bool = False, stream=None) -> dict:
    import torch

    f, keep = make_field(field)
    nblk = 1
    for k in range(f.ndim):
        nblk *= (f.shape[k] + 3) // 4
    nb = 4 ** f.ndim
    dev = torch.device("cuda")
    emax = torch.zeros(nblk, dtype=torch.int32, device=dev)
    prec = torch.zeros(nblk, dtype=torch.int32, device=dev)
    bits = torch.zeros(nblk, dtype=torch.int64, device=dev)
    coeffs = torch.zeros(nblk * nb, dtype=torch.int32, device=dev) if want_coeffs else None
    _check(lib().rd_zfp_blocks(ctx, C.byref(f), float(eb_abs), _ptr(emax), _ptr(prec), _ptr(bits),
                               _ptr(coeffs), _stream(stream)), "rd_zfp_blocks")
    out = {"emax": emax.cpu().numpy(), "prec": prec.cpu().numpy(),
           "bits": bits.cpu().numpy().view(np.uint64)}
    if want_coeffs:
        out["coeffs"] = coeffs.cpu().numpy().view(np.uint32).reshape(nblk, nb)
    return out


def rd_sz_symbols(ctx, field, delta: float, quant_radius: int = 32768, strides=None,
                  stream=None) -> dict:
    import torch

    f, keep = make_field(field)
    n = 1
    for k in range(f.ndim):
        n *= f.shape[k]
    dev = torch.device("cuda")
    est = torch.empty(n, dtype=torch.int32, device=dev)
    gt = torch.empty(n, dtype=torch.int32, device=dev)
    rec = torch.empty(n, dtype=torch.float32, device=dev)
    st = None
    if strides is not None:
        st = np.array(list(strides), dtype=np.int32)
    _check(lib().rd_sz_symbols(ctx, C.byref(f), float(delta), int(quant_radius), _ptr(st),
                               _ptr(est), _ptr(gt), _ptr(rec), _stream(stream)), "rd_sz_symbols")
    shape = tuple(f.shape[k] for k in range(f.ndim))
    return {"est": est.cpu().numpy().reshape(shape), "gt": gt.cpu().numpy().reshape(shape),
            "recon": rec.cpu().numpy().reshape(shape)}


def rd_set_profiling(ctx, on: bool) -> None:
    _check(lib().rd_set_profiling(ctx, 1 if on else 0), "rd_set_profiling")


def rd_reset_profile(ctx) -> None:
    _check(lib().rd_reset_profile(ctx), "rd_reset_profile")


def rd_kernel_stats(ctx) -> dict:
    """{kernel name: (total ms, launches)} from rd_kernel_stat."""
    out, i = {}, 0
    name, ms, n = C.c_char_p(), C.c_double(), C.c_int64()
    while lib().rd_kernel_stat(ctx, i, C.byref(name), C.byref(ms), C.byref(n)) == RD_OK:
        out[name.value.decode()] = (ms.value, n.value)
        i += 1
    return out


def rd_launch_count(ctx) -> int:
    return int(lib().rd_launch_count(ctx))


class Server:
    """Owns one rd_server (the serving loop).  submit() keeps a reference to
    the field until its completion has been polled, since the library reads
    the field's memory while the request is pending or running."""

    def __init__(self, device: int = 0, slots: int = 4, window: int = 8, hbm_budget: int = 0):
        cfg = rd_server_config(int(device), int(slots), int(window), 0, int(hbm_budget))
        h = C.c_void_p()
        _check(lib().rd_server_create(C.byref(cfg), C.byref(h)), "rd_server_create")
        self.h = h
        self._keep = {}

    def submit(self, x, prm: rd_params, key: int = 0, tag: int = 0) -> int:
        f, keep = make_field(x)
        rid = C.c_uint64()
        _check(lib().rd_server_submit(self.h, C.byref(f), C.byref(prm), int(key), int(tag),
                                      C.byref(rid)), "rd_server_submit")
        self._keep[rid.value] = (keep, prm)
        return rid.value

    def poll(self, max_n: int = 256, wait_ms: int = 0) -> list:
        buf = (rd_server_completion * max_n)()
        n = C.c_int32()
        _check(lib().rd_server_poll(self.h, buf, int(max_n), int(wait_ms), C.byref(n)),
               "rd_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            self._keep.pop(c.request_id, None)
            d = {k: getattr(c, k) for k, _ in rd_server_completion._fields_ if k != "result"}
            d["result"] = _todict(c.result)
            out.append(d)
        return out

    def stats(self) -> dict:
        st = rd_server_stats()
        _check(lib().rd_server_get_stats(self.h, C.byref(st)), "rd_server_get_stats")
        return _todict(st)

    def reset_stats(self) -> None:
        _check(lib().rd_server_reset_stats(self.h), "rd_server_reset_stats")

    def close(self):
        if self.h:
            _check(lib().rd_server_destroy(self.h), "rd_server_destroy")
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owns one rd_context; methods forward to the entry points above."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.h = rd_context_create(device, hbm_budget)

    def close(self):
        if self.h:
            rd_context_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def estimate_zfp(self, x, p, stream=None):
        return rd_estimate_zfp(self.h, x, p, stream)

    def estimate_sz(self, x, p, delta=0.0, stream=None):
        return rd_estimate_sz(self.h, x, p, delta, stream)

    def estimate_sz_log(self, x, p, stream=None):
        return rd_estimate_sz_log(self.h, x, p, stream)

    def select(self, x, p, stream=None):
        return rd_select(self.h, x, p, stream)

    def ground_truth(self, x, p, eb_sz=0.0, stream=None):
        return rd_ground_truth(self.h, x, p, eb_sz, stream)

    def zfp_compress(self, x, p, out=None, stream=None):
        return rd_zfp_compress(self.h, x, p, out, stream)

    def compress(self, x, p, out=None, stream=None):
        return rd_compress(self.h, x, p, out, stream)

    def sz_compress(self, x, p, eb_sz, out=None, stream=None):
        return rd_sz_compress(self.h, x, p, eb_sz, out, stream)

    def ground_truth_classic(self, x, p, eb_sz, recon=None, stream=None):
        return rd_ground_truth_classic(self.h, x, p, eb_sz, recon, stream)

    def evaluate(self, x, p, stream=None):
        return rd_evaluate(self.h, x, p, stream)

    def rd_curve(self, x, p, ebs, stream=None):
        return rd_rd_curve(self.h, x, p, ebs, stream)

    def select_batch(self, fields, prms, truth=False, stream=None, check=True):
        return rd_select_batch(self.h, fields, prms, truth, stream, check)

    def batch_call(self, fields, prms, truth=False):
        return BatchCall(self.h, fields, prms, truth)

    def batch_set_config(self, cfg=None):
        rd_batch_set_config(self.h, cfg)

    def batch_get_config(self):
        return rd_batch_get_config(self.h)

    def histograms(self):
        return rd_copy_histograms(self.h)

    def zfp_blocks(self, x, eb_abs, want_coeffs=False, stream=None):
        return rd_zfp_blocks(self.h, x, eb_abs, want_coeffs, stream)

    def sz_symbols(self, x, delta, quant_radius=32768, strides=None, stream=None):
        return rd_sz_symbols(self.h, x, delta, quant_radius, strides, stream)

    def set_profiling(self, on=True):
        rd_set_profiling(self.h, on)

    def reset_profile(self):
        rd_reset_profile(self.h)

    def kernel_stats(self):
        return rd_kernel_stats(self.h)

    def launch_count(self):
        return rd_launch_count(self.h)
