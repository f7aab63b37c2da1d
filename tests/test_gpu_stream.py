"""The SZ stream written on the GPU (rd_sz_compress) against the oracle: its
length is the ground truth's bit count, and the oracle's decoder reads back
from it every point's symbol (the oracle's prequantised symbols) and every
escaped value, bit for bit.  Equal-weight ties of the Huffman tree may be
broken differently on the two sides, so the streams are compared through
decoding, not byte by byte; the payload length is the same for every
optimal code."""
import numpy as np
import pytest

import synth

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_08901_gb300 import _build, rdsel

    _build.build()
    return rdsel


@pytest.fixture(scope="module")
def ctx(R):
    c = R.Context(0)
    yield c
    c.close()


def _gp(R, op):
    return R.params(eb=op.eb, eb_mode=op.eb_mode, ec_mode=op.ec_mode, r_sp=op.r_sp,
                    quant_radius=op.quant_radius, sel_rule=op.sel_rule, sz_offset=op.sz_offset)


def _fields():
    rng = np.random.default_rng(11)
    f = {}
    f["1d_ragged"] = (synth.grf_np((4097,), -2.0, 11) * 3).astype(np.float32)
    f["2d_ragged"] = (synth.grf_np((61, 58), -3.0, 12) * 50 + 7).astype(np.float32)
    f["3d_ragged"] = (synth.grf_np((17, 22, 19), -3.0, 13) * 2).astype(np.float32)
    f["3d_noise"] = rng.standard_normal((12, 16, 20)).astype(np.float32)
    f["2d_fill"] = synth.fill_region_np(synth.grf_np((48, 64), -3.0, 15), seed=16)
    f["3d_large"] = synth.config2_field(seed=4, shape=(40, 100, 100))
    return f


FIELDS = _fields()


def compress(R, ctx, x, op, eb_sz):
    xd = torch.from_numpy(x).cuda()
    gp = _gp(R, op)
    nbits = ctx.sz_compress(xd, gp, eb_sz)
    out = torch.full((8 * ((nbits + 63) // 64),), 0xA5, dtype=torch.uint8, device="cuda")
    assert ctx.sz_compress(xd, gp, eb_sz, out) == nbits
    return nbits, out.cpu().numpy()


@pytest.mark.parametrize("name", sorted(FIELDS))
@pytest.mark.parametrize("rel_eb,radius", [(1e-3, 32768), (1e-5, 32768), (1e-3, 8)])
def test_stream_decodes_to_the_oracle_symbols(R, ctx, name, rel_eb, radius):
    x = FIELDS[name]
    vr = float(x.max()) - float(x.min())
    eb_sz = rel_eb * vr
    op = O.params(eb=1e-3, quant_radius=radius)
    nbits, buf = compress(R, ctx, x, op, eb_sz)
    t = O.ground_truth(x, op, eb_sz)
    assert nbits == t["sz_bits_gt"]
    # the bytes past the last bit are zero
    nbytes = (nbits + 7) // 8
    assert not buf[nbytes:].any()
    if nbits % 8:
        assert buf[nbytes - 1] & ((1 << (8 - nbits % 8)) - 1) == 0
    sym, esc = O.sz_stream_decode(buf[:nbytes].tobytes(), nbits, x.size)
    ref = O.sz_symbols(x, 2 * eb_sz, quant_radius=radius)["gt"].ravel()
    assert np.array_equal(sym, ref)
    assert np.array_equal(esc.view(np.uint32), x.ravel()[ref == 0].view(np.uint32))
    if radius == 8:
        assert t["sz_nesc_gt"] > 0


def test_stream_errors(R, ctx):
    x = FIELDS["2d_ragged"]
    xd = torch.from_numpy(x).cuda()
    gp = _gp(R, O.params(eb=1e-3))
    nbits = ctx.sz_compress(xd, gp, 0.01)
    words = (nbits + 63) // 64
    small = torch.zeros(8 * words - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.sz_compress(xd, gp, 0.01, small)
    assert e.value.code == R.RD_ERR_RANGE
    big = torch.zeros(8 * words + 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.sz_compress(xd, gp, 0.01, big[1:])  # not 8-byte aligned
    assert e.value.code == R.RD_ERR_INVALID_ARG
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(R.RdselError) as e:
            ctx.sz_compress(xd, gp, bad)
        assert e.value.code == R.RD_ERR_INVALID_ARG
    const = torch.full((9, 13), 2.0, dtype=torch.float32, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.sz_compress(const, gp, 0.01)
    assert e.value.code == R.RD_ERR_INVALID_ARG


def test_stream_of_a_host_field_and_repeats(R, ctx):
    """A host field (staged) gives the same stream as the device copy, and a
    repeated call the same bytes."""
    x = FIELDS["3d_ragged"]
    op = O.params(eb=1e-3)
    gp = _gp(R, op)
    nbits = ctx.sz_compress(x, gp, 0.005)
    out_h = torch.zeros(8 * ((nbits + 63) // 64), dtype=torch.uint8, device="cuda")
    ctx.sz_compress(x, gp, 0.005, out_h)
    n2, buf = compress(R, ctx, x, op, 0.005)
    assert n2 == nbits and np.array_equal(out_h.cpu().numpy(), buf)
    n3, buf3 = compress(R, ctx, x, op, 0.005)
    assert n3 == nbits and np.array_equal(buf3, buf)


def _table(buf, nbits):
    """The header and code table of a stream: K, escapes, and per present
    symbol (ascending) its code length."""
    bits = np.unpackbits(np.frombuffer(buf, dtype=np.uint8))
    def field(p, n):
        return int("".join(map(str, bits[p:p + n])), 2) if n else 0
    K, nesc = field(0, 32), field(32, 32)
    lens = {}
    for r in range(K):
        lens[field(64 + 22 * r, 16)] = field(64 + 22 * r + 16, 6)
    return K, nesc, lens


@pytest.mark.parametrize("shape,rel_eb", [((64, 128, 256), 1e-6), ((40, 100, 100), 1e-4),
                                          ((4096,), 1e-2)])
def test_code_table_built_on_the_device(R, ctx, shape, rel_eb):
    """The code table is built on the device: the same bytes on every call,
    an optimal code (the lengths' weighted sum is the Huffman cost, the
    Kraft sum is at most one), the table in ascending symbol order with the
    histogram's symbols; the widest case has more symbols than the shared-
    memory queues hold (the queues go to global memory), the last a handful
    of symbols."""
    x = (synth.grf_np(shape, -1.5, 91) * 7).astype(np.float32)
    vr = float(x.max()) - float(x.min())
    eb_sz = rel_eb * vr
    op = O.params(eb=1e-3)
    nbits, buf = compress(R, ctx, x, op, eb_sz)
    nbits2, buf2 = compress(R, ctx, x, op, eb_sz)
    assert nbits2 == nbits and np.array_equal(buf, buf2)
    t = O.ground_truth(x, op, eb_sz, want_hist=True)
    h = np.asarray(t["hist"], dtype=np.int64)
    K, nesc, lens = _table(buf[: (nbits + 7) // 8].tobytes(), nbits)
    assert K == t["sz_nsym_gt"] == int((h > 0).sum()) and nesc == t["sz_nesc_gt"]
    assert sorted(lens) == list(np.nonzero(h)[0])
    assert sum(int(h[s]) * L for s, L in lens.items()) == t["sz_huff_gt"]
    if K > 1:
        assert sum(2.0 ** -L for L in lens.values()) <= 1.0
    if shape == (64, 128, 256):
        assert K > 28672
    sym, _ = O.sz_stream_decode(buf[: (nbits + 7) // 8].tobytes(), nbits, x.size)
    assert np.array_equal(sym, O.sz_symbols(x, 2 * eb_sz)["gt"].ravel())
