"""rd_select_static: the estimate for callers that may not allocate memory.

Some callers cannot call cudaMalloc: an in-situ simulation that owns the
GPU's memory budget, a framework whose allocator must serve every allocation,
code that cannot take the synchronisation an allocation may imply.  For them
rd_select_static runs rd_select's kernels on a fixed scratch array inside the
library.  This test calls it through the C ABI twice in a row on each field
and checks both results against rd_select (bit-exact integers and singly
rounded doubles; entropy and PSNR within the suite's tolerances), and that it
refuses what it cannot serve without allocating.

This file is collected last on purpose; it also passes alone in a fresh
process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL_PSNR = 1e-6
REL_ENTROPY = 1e-10
EXACT = ["vmin", "vmax", "vr", "eb_abs", "r_sp_eff", "strides", "minexp", "n_blocks",
         "n_sampled_blocks", "zfp_s2", "zfp_npoints", "zfp_ncoeff", "mse_sp", "br_zfp",
         "delta", "sz_ns", "sz_huff_bits", "sz_nesc", "sz_nsym", "br_sz_huff", "selection",
         "flags"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_08901_gb300 import _build, rdsel

    _build.build()
    return rdsel


def _rel(a, b):
    return 0.0 if a == b else abs(a - b) / max(abs(a), abs(b))


def _same(a, b):
    for k in EXACT:
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("psnr_zfp", "psnr_sz"):
        assert _rel(a[k], b[k]) <= REL_PSNR, k
    for k in ("entropy", "br_sz"):
        assert _rel(a[k], b[k]) <= REL_ENTROPY, k


@pytest.mark.parametrize("shape,eb,r_sp", [
    ((24, 40, 44), 1e-4, 0.05),
    ((61, 58), 1e-3, 1.0),
    ((4097,), 1e-5, 0.2),
])
def test_static_select_matches_rd_select_twice(R, shape, eb, r_sp):
    if len(shape) == 3:
        x = synth.config2_field(seed=21, shape=shape)
    else:
        x = (synth.grf_np(shape, -3.0, 22) * 10).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    p = R.params(eb=eb, r_sp=r_sp)
    with R.Context(0) as ctx:
        ref = ctx.select(xd, p)
    first = R.rd_select_static(xd, p)
    second = R.rd_select_static(xd, p)  # the scratch keeps the last call's contents
    _same(first, ref)
    _same(second, ref)


def test_static_select_after_other_field(R):
    """A call on a different field in between must not leak into the next."""
    a = torch.from_numpy(synth.config1_field(seed=23, shape=(64, 64))).cuda()
    b = torch.from_numpy(synth.config2_field(seed=24, shape=(12, 16, 20))).cuda()
    p = R.params(eb=1e-3, r_sp=0.25)
    with R.Context(0) as ctx:
        ra, rb = ctx.select(a, p), ctx.select(b, p)
    _same(R.rd_select_static(a, p), ra)
    _same(R.rd_select_static(b, p), rb)
    _same(R.rd_select_static(a, p), ra)


def test_static_select_refuses_what_needs_allocation(R):
    x = synth.config1_field(seed=25, shape=(32, 32))
    p = R.params()
    with pytest.raises(R.RdselError) as e:
        R.rd_select_static(x, p)  # host array: would need a staging buffer
    assert e.value.code == R.RD_ERR_INVALID_ARG
    # more than 2^31 - 1 points
    xd = torch.from_numpy(x).cuda()
    f = R.rd_field(xd.data_ptr(), 3, R.RD_LOC_DEVICE, (C.c_int64 * 3)(65536, 65536, 2))
    r = R.rd_result()
    rc = R.lib().rd_select_static(C.byref(f), C.byref(p), C.byref(r), None)
    assert rc == R.RD_ERR_INVALID_ARG


def test_static_select_leaves_device_memory_untouched(R):
    """The device's free memory is the same before and after a run of calls
    on a large field (after one warm-up call): nothing was allocated.  The
    reading is repeated a few times, since another process on the GPU could
    move it; a slack of 2 MiB covers the driver's own bookkeeping."""
    x = torch.from_numpy(synth.config2_field(seed=26, shape=(64, 256, 256))).cuda()
    p = R.params(eb=1e-4, r_sp=0.05)
    R.rd_select_static(x, p)
    torch.cuda.synchronize()
    ok = False
    for _ in range(3):
        free0, _total = torch.cuda.mem_get_info()
        for _ in range(8):
            R.rd_select_static(x, p)
        torch.cuda.synchronize()
        free1, _total = torch.cuda.mem_get_info()
        if abs(free1 - free0) <= (2 << 20):
            ok = True
            break
    assert ok, (free0, free1)
