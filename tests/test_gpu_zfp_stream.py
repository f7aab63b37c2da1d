"""The ZFP fixed-accuracy stream written on the GPU (rd_zfp_compress) and
Algorithm 1 to the end (rd_compress: the selection s_i, then the selected
compressor's bytes C_i), against the oracle.

The ZFP stream has no free choice (blocks in order, group tests as the
planes decide them), so it is compared with the oracle's encoder byte for
byte; its length is the ZFP truth's bit count, and the oracle's decoder
rebuilds the field from the GPU's bytes within eb_abs.  An SZ stream chosen
by rd_compress is read back by the oracle's decoder (equal-weight ties of a
Huffman tree may be broken either way, so SZ streams are compared through
decoding)."""
import numpy as np
import pytest

import synth
from test_gpu_parity import R, ctx, _gp  # noqa: F401

O = pytest.importorskip("oracle")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _fields():
    rng = np.random.default_rng(21)
    f = {}
    f["1d_ragged"] = (synth.grf_np((4097,), -2.0, 71) * 3).astype(np.float32)
    f["2d_ragged"] = (synth.grf_np((61, 58), -3.0, 72) * 50 + 7).astype(np.float32)
    f["3d_ragged"] = (synth.grf_np((17, 22, 19), -3.0, 73) * 2).astype(np.float32)
    f["3d_noise"] = rng.standard_normal((12, 16, 20)).astype(np.float32)
    f["2d_fill"] = synth.fill_region_np(synth.grf_np((48, 64), -3.0, 74), seed=75)
    f["3d_large"] = synth.config2_field(seed=76, shape=(40, 100, 100))
    return f


FIELDS = _fields()


def _zfp(R, ctx, xd, gp):
    nbits = ctx.zfp_compress(xd, gp)
    out = torch.full((8 * ((nbits + 63) // 64),), 0xA5, dtype=torch.uint8, device="cuda")
    assert ctx.zfp_compress(xd, gp, out) == nbits
    return nbits, out.cpu().numpy()


@pytest.mark.parametrize("name", sorted(FIELDS))
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_zfp_stream_equals_the_oracle_stream(R, ctx, name, eb):
    x = FIELDS[name]
    op = O.params(eb=eb)
    xd = torch.from_numpy(x).cuda()
    nbits, buf = _zfp(R, ctx, xd, _gp(R, op))
    t = O.ground_truth(x, op)
    assert nbits == t["zfp_bits_gt"]
    eb_abs = O.select(x, op)["eb_abs"]
    data, onbits = O.zfp_stream(x, eb_abs)
    assert onbits == nbits
    nbytes = (nbits + 7) // 8
    assert buf[:nbytes].tobytes() == data
    assert not buf[nbytes:].any()
    rec = O.zfp_stream_decode(buf[:nbytes].tobytes(), nbits, x.shape, eb_abs)
    err = np.abs(rec.astype(np.float64) - x.astype(np.float64)).max()
    assert err == t["maxerr_zfp"]


def test_zfp_stream_every_plane_and_empty_blocks(R, ctx):
    """Blocks that code all 32 planes (a bound far below the values) and
    blocks that code none (a fill region at 1e-20 next to values of order
    one), ragged edges."""
    x = (synth.grf_np((13, 18, 22), -3.0, 77) * 200 + 1000).astype(np.float32)
    op = O.params(eb=1e-9, eb_mode=O.EB_ABS)
    nbits, buf = _zfp(R, ctx, torch.from_numpy(x).cuda(), _gp(R, op))
    data, onbits = O.zfp_stream(x, 1e-9)
    assert nbits == onbits and buf[: (nbits + 7) // 8].tobytes() == data
    y = FIELDS["2d_fill"]
    op = O.params(eb=1e-3)
    nbits, buf = _zfp(R, ctx, torch.from_numpy(y).cuda(), _gp(R, op))
    data, onbits = O.zfp_stream(y, O.select(y, op)["eb_abs"])
    assert nbits == onbits and buf[: (nbits + 7) // 8].tobytes() == data


def test_zfp_stream_errors_and_host_field(R, ctx):
    x = FIELDS["3d_ragged"]
    gp = _gp(R, O.params(eb=1e-3))
    nbits = ctx.zfp_compress(x, gp)  # host field: staged
    words = (nbits + 63) // 64
    small = torch.zeros(8 * words - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.zfp_compress(x, gp, small)
    assert e.value.code == R.RD_ERR_RANGE
    big = torch.zeros(8 * words + 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.zfp_compress(x, gp, big[1:])
    assert e.value.code == R.RD_ERR_INVALID_ARG
    const = torch.full((9, 13), 2.0, dtype=torch.float32, device="cuda")
    with pytest.raises(R.RdselError) as e:
        ctx.zfp_compress(const, gp)
    assert e.value.code == R.RD_ERR_INVALID_ARG
    out = torch.zeros(8 * words, dtype=torch.uint8, device="cuda")
    ctx.zfp_compress(x, gp, out)
    _, buf = _zfp(R, ctx, torch.from_numpy(x).cuda(), gp)
    assert np.array_equal(out.cpu().numpy(), buf)


@pytest.mark.parametrize("name,eb,r_sp", [("3d_large", 1e-4, 0.05), ("2d_ragged", 1e-2, 1.0),
                                          ("3d_noise", 1e-3, 0.25), ("1d_ragged", 1e-5, 0.2),
                                          ("2d_fill", 1e-4, 0.05)])
def test_compress_writes_the_selected_stream(R, ctx, name, eb, r_sp):
    """rd_compress: s_i is the oracle's selection; C_i is ZFP's stream at
    eb_abs (byte for byte) when s_i = 1, SZ's at eb_sz = delta / 2 (read back
    by the oracle's decoder) when s_i = 0."""
    x = FIELDS[name]
    op = O.params(eb=eb, r_sp=r_sp)
    xd = torch.from_numpy(x).cuda()
    gp = _gp(R, op)
    o = O.select(x, op)
    size = ctx.compress(xd, gp)
    assert size["selection"] == o["selection"]
    out = torch.zeros(8 * ((size["nbits"] + 63) // 64), dtype=torch.uint8, device="cuda")
    got = ctx.compress(xd, gp, out)
    assert got["selection"] == o["selection"] and got["nbits"] == size["nbits"]
    assert got["est"]["delta"] == o["delta"]
    nbits = got["nbits"]
    buf = out.cpu().numpy()[: (nbits + 7) // 8].tobytes()
    if got["selection"] == 1:
        data, onbits = O.zfp_stream(x, o["eb_abs"])
        assert nbits == onbits and buf == data
    else:
        eb_sz = o["delta"] / 2
        t = O.ground_truth(x, op, eb_sz)
        assert nbits == t["sz_bits_gt"]
        sym, esc = O.sz_stream_decode(buf, nbits, x.size)
        ref = O.sz_symbols(x, o["delta"])["gt"].ravel()
        assert np.array_equal(sym, ref)


def test_compress_selects_both_compressors(R, ctx):
    """Over the fields and bounds above, both outcomes of the selection
    occur, so both stream paths of rd_compress are exercised."""
    seen = set()
    for name in ("3d_large", "2d_ragged", "3d_noise", "1d_ragged", "2d_fill"):
        for eb in (1e-2, 1e-4, 1e-6):
            seen.add(O.select(FIELDS[name], O.params(eb=eb))["selection"])
    assert seen == {0, 1}
