"""8-bit UNORM outputs (NTC_DTYPE_U8): each output y is stored as
rn(clamp(y, 0, 1) * 255) in float32 (ties to even, NaN -> 0).

The integer is decided in float32 on both sides: every path's U8 output must
equal, bit for bit, that rounding of the same path's float32 output (the
kernels compute y identically for both output types and differ only in the
store).  Against the FP64 oracle the bar is one code: the float outputs are
within 2e-3 (0.51 of a code) of the oracle, so the rounded codes can differ
by at most 1.
"""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def unorm8(y: torch.Tensor) -> torch.Tensor:
    """rn(sat(y) * 255) with the product rounded to float32 first."""
    y = torch.nan_to_num(y.float(), nan=0.0).clamp(0.0, 1.0) * 255.0
    return torch.round(y).to(torch.uint8)


def _f8(mat16, case):
    """E4M3 weights with per-layer scales (max |w| -> 448), activation scales
    1/256, 4/256, 4/256."""
    ws, q8 = [], []
    for w in case.weights[0::2]:
        s = float(np.abs(w).max()) / 448.0
        ws.append(s)
        q8.append(torch.from_numpy(w / s).to(DEV).to(torch.float8_e4m3fn).view(torch.uint8))
    scale = torch.tensor(ws + [1.0 / 256, 4.0 / 256, 4.0 / 256], dtype=torch.float32, device=DEV)
    return mat16.with_(weights=q8, precision=ntc.PREC_F8, scale=scale)


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


SHAPES = [
    dict(width=512, height=512, channels=16, c0=12, c1=12, k_in=48),   # fast class, 16-byte rows
    dict(width=256, height=256, channels=12, c0=16, c1=16, k_in=48),   # 4-byte words
    dict(width=256, height=256, channels=8, c0=8, c1=8, k_in=32),
    dict(width=128, height=64, channels=5, c0=3, c1=6, bits0=2, bits1=8, k_in=32, act=1),
    dict(width=128, height=128, channels=3, c0=14, c1=10, k_in=48),    # scalar bytes
    dict(width=64, height=64, channels=16, c0=12, c1=12, k_in=64, out_act=1),  # outside [0, 1]
    dict(width=256, height=256, channels=12, c0=12, c1=12, q0=0.1, q1=0.05, k_in=48),  # generic
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("form", ["simt", "ws", "nwg4", "f8"])
def test_u8_is_unorm_of_f32_output(shape, form):
    case = make_case(seed=301, **shape)
    if form == "f8" and case.k_in % 32:
        pytest.skip("FP8 operands need K a multiple of 32")
    mat, md = device_material(case, precision=ntc.PREC_F32 if form == "simt" else ntc.PREC_F16)
    if form == "f8":
        mat = _f8(mat, case)
    q = gen.random_queries(9 * 128 + 77, md.mips, seed=4301)
    q[:2] = [[0.0, 0.0, 0.0], [0.999999, 0.999999, md.mips - 1]]
    uvl = _uvl(q)
    ntc.ntc_set_decode_warpgroups(4 if form == "nwg4" else 0)
    try:
        for filt in (ntc.FILTER_NEAREST, ntc.FILTER_TRILINEAR, ntc.FILTER_STOCHASTIC):
            kw = dict(filter=filt, noise_seed=7, noise_step=3)
            y = ntc.ntc_decode(mat, uvl, out_dtype=torch.float32, **kw)
            u = ntc.ntc_decode(mat, uvl, out_dtype=torch.uint8, **kw)
            assert ntc.ntc_device_status() == ntc.OK
            assert u.dtype == torch.uint8 and u.shape == y.shape
            assert torch.equal(u, unorm8(y)), (form, filt)
    finally:
        ntc.ntc_set_decode_warpgroups(0)


@pytest.mark.parametrize("shape", SHAPES[:5])
def test_u8_within_one_code_of_oracle(shape):
    case = make_case(seed=302, **shape)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = gen.random_queries(7 * 128 + 45, md.mips, seed=4302)
    ref = np.rint(np.clip(md.decode(q), 0.0, 1.0) * 255.0)
    got = ntc.ntc_decode(mat, _uvl(q), out_dtype=torch.uint8).cpu().numpy().astype(np.int64)
    assert np.abs(got - ref).max() <= 1
    # the FP32 CUDA-core form is within 1e-5 of the oracle: codes agree except
    # where the oracle's value sits within 1e-5 of a rounding boundary
    mat32, md32 = device_material(case, precision=ntc.PREC_F32)
    got32 = ntc.ntc_decode(mat32, _uvl(q), out_dtype=torch.uint8).cpu().numpy().astype(np.int64)
    code = np.clip(md32.decode(q), 0.0, 1.0) * 255.0
    near = np.abs(code - np.floor(code) - 0.5) < 255 * 1e-5
    assert np.array_equal(got32[~near], np.rint(code)[~near])


@pytest.mark.parametrize("filt", [ntc.FILTER_NEAREST, ntc.FILTER_TRILINEAR])
def test_batched_u8_unaligned_output_blocks(filt):
    """Output blocks of 3-, 5- and 7-channel materials start at byte offsets
    that are not 16-byte aligned: the batched kernel stores those bytes one
    by one and the aligned ones as vectors."""
    specs = [(128, 3, 8, 8), (256, 16, 12, 12), (64, 5, 16, 16), (128, 7, 8, 16), (256, 12, 13, 10),
             (128, 16, 12, 12)]
    mats, qs = [], []
    for i, (side, c, c0, c1) in enumerate(specs):
        case = make_case(side, side, c, c0, c1, k_in=48, seed=310 + i)
        mats.append(device_material(case, precision=ntc.PREC_F16))
        qs.append(gen.random_queries(131 * (i + 1) + 3, oracle.mips(side, side), seed=4310 + i))
    batch = ntc.Batch([m for m, _ in mats], [len(q) for q in qs], filter=filt)
    uvl = _uvl(np.concatenate(qs))
    y = ntc.ntc_decode_batched(batch, uvl, out_dtype=torch.float32)
    u = ntc.ntc_decode_batched(batch, uvl, out_dtype=torch.uint8)
    assert ntc.ntc_device_status() == ntc.OK
    assert any(int(o) % 16 for o in batch.o_offsets[:-1])
    assert torch.equal(u, unorm8(y))
    # the batched kernel's floats are within 1e-6 of the single-material decode
    for i, (m, _) in enumerate(mats):
        single = ntc.ntc_decode(m, _uvl(qs[i]), out_dtype=torch.uint8, filter=filt)
        blk = u[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(qs[i]), m.channels)
        assert (blk.int() - single.int()).abs().max() <= 1, i


@pytest.mark.parametrize("chunk", [128, 1 << 12])
def test_decode_host_u8(chunk):
    case = make_case(512, 512, 12, 12, 12, k_in=48, seed=320)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = torch.from_numpy(gen.random_queries(9 * 1024 + 13, md.mips, seed=4320)).pin_memory()
    ref = ntc.ntc_decode(mat, q.to(DEV), out_dtype=torch.uint8).cpu()
    ws = torch.empty(ntc.lib().ntc_decode_host_workspace_bytes(mat.channels, ntc.DTYPE_U8, chunk),
                     dtype=torch.uint8, device=DEV)
    out = ntc.ntc_decode_host(mat, q, out_dtype=torch.uint8, workspace=ws)
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    assert out.dtype == torch.uint8 and torch.equal(out, ref)
