"""Vector-quantised G0 (the paper's comparison with vector quantisation,
VQ-8 and VQ-16: two 256-entry codebooks, two 8-bit indices per cell, a cell's
features the sum of its two entries): the GPU encoder's indices bit-exact
against the oracle's greedy residual search, and decode (FP32 and FP16
forms, nearest and trilinear, bilinear and learned G0) against the oracle
of the reconstructed grids."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material, to_np

pytestmark = pytest.mark.gpu
OUT_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _codebooks(books, c0, seed):
    rng = np.random.default_rng(seed)
    cb = rng.uniform(-0.5, 0.5, (books, 256, c0)).astype(np.float32)
    cb[1:] *= 0.25                      # later books refine the first
    return cb


@pytest.mark.parametrize("books,c0", [(1, 8), (2, 8), (2, 16), (4, 5)])
def test_vq_assign_bit_exact(books, c0):
    rng = np.random.default_rng(100 + c0)
    vals = rng.uniform(-0.6, 0.6, (3 * 4096 + 17, c0)).astype(np.float32)
    cb = _codebooks(books, c0, 200 + c0)
    got = ntc.ntc_vq_assign(torch.from_numpy(vals).to(DEV), torch.from_numpy(cb).to(DEV))
    assert np.array_equal(got.cpu().numpy(), oracle.vq_assign(vals, cb))


def _vq_material(case, books, precision, seed):
    """The case's G0 replaced by a vector-quantised one: indices assigned to
    the case's own G0 values by the library's encoder, the oracle fed the
    reconstruction of the same indices."""
    cb = _codebooks(books, case.c0, seed)
    mat, md = device_material(case, precision=precision)
    idx = [ntc.ntc_vq_assign(torch.from_numpy(v.reshape(-1, case.c0)).to(DEV),
                             torch.from_numpy(cb).to(DEV)).reshape(v.shape[0], v.shape[1], books)
           for v in case.val0]
    g0 = [oracle.vq_reconstruct(i.cpu().numpy(), cb) for i in idx]
    m = mat.with_(grids0=idx, codebook0=torch.from_numpy(cb).to(DEV))
    md_vq = oracle.Model(case.width, case.height, case.channels, case.c0, case.c1, case.n0,
                         case.n1, case.q0, case.q1, g0, md.grids1, md.weights, case.k_in,
                         act=case.act, out_act=case.out_act, interp0=case.interp0)
    return m, md_vq


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
@pytest.mark.parametrize("shape,books", [
    (dict(width=512, height=512, channels=16, c0=8, c1=12, k_in=48), 2),        # VQ-8
    (dict(width=256, height=256, channels=9, c0=16, c1=12, k_in=48), 2),        # VQ-16
    (dict(width=256, height=128, channels=6, c0=8, c1=12, k_in=64, act=1, out_act=1,
          interp0=1), 2),                                                        # learned G0
])
def test_vq_decode_matches_oracle(shape, books, precision):
    case = make_case(seed=87, **shape)
    mat, md = _vq_material(case, books, precision, 300)
    assert mat.struct.vq_books == books
    q = gen.random_queries(3 * 4096 + 7, md.mips, seed=4087)
    out = to_np(ntc.ntc_decode(mat, torch.from_numpy(q).to(DEV)))
    assert ntc.ntc_device_status() == ntc.OK
    assert np.abs(out - md.decode(q)).max() <= OUT_TOL
    tri = to_np(ntc.ntc_decode(mat, torch.from_numpy(q[:1500]).to(DEV), filter=ntc.FILTER_TRILINEAR))
    assert np.abs(tri - md.decode_trilinear(q[:1500])).max() <= OUT_TOL


def test_vq_refusals():
    case = make_case(seed=88, width=256, height=256, channels=8, c0=8, c1=8, k_in=32)
    mat, _ = _vq_material(case, 2, ntc.PREC_F16, 301)
    q = torch.from_numpy(gen.random_queries(256, case.mips, seed=4088)).to(DEV)
    with pytest.raises(ntc.NTCError):
        ntc.ntc_decode(mat, q, flags=ntc.FLAG_NOISE)
    with pytest.raises(ntc.NTCError):
        ntc.Batch([mat], [256], ntc.FILTER_NEAREST)
