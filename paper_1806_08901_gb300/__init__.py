"""GB300-native online rate-distortion estimation and SZ-vs-ZFP selection
(Tao et al., arXiv 1806.08901).

The product is ``librdsel.so`` (C ABI in include/rdsel.h, hand-written CUDA
for sm_103a); ``rdsel`` is its thin ctypes binding.  Build it with
``paper_1806_08901_gb300._build.build()``.
"""
from . import rdsel  # noqa: F401
from .rdsel import (  # noqa: F401
    Context, RdselError, RdselUnavailable, params,
    rd_context_create, rd_context_destroy, rd_estimate_zfp, rd_estimate_sz, rd_select,
    rd_ground_truth, rd_evaluate, rd_copy_histograms, rd_zfp_blocks, rd_sz_symbols,
    RD_EB_REL, RD_EB_ABS, RD_EC_PAPER, RD_EC_ALL, RD_SEL_PAPER, RD_SEL_HUFFMAN,
)
