"""Vector-quantised G0 (the paper's comparison with vector quantisation,
VQ-8 and VQ-16: two 256-entry codebooks, two 8-bit indices per cell, a cell's
features the sum of its two entries): the GPU encoder's indices bit-exact
against the oracle's greedy residual search, decode (FP32 and FP16 forms,
nearest and trilinear, bilinear and learned G0) against the oracle of the
reconstructed grids, and the training step of a vector-quantised G0 (VQ-VAE
terms) against the oracle's."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, check_grads, device_material, rel_err, to_np

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


@pytest.mark.parametrize("nwg", [2, 4, 5])
def test_vq_fast_layout_every_launch_shape(nwg):
    """VQ-8 with a 4-bit G1 runs the fast layout (FP16 codebooks in shared
    memory, exact bilinear weights on the 1/16 lattice) on every launch
    shape: against the oracle, nearest and trilinear."""
    case = make_case(seed=86, width=512, height=256, channels=12, c0=8, c1=12, k_in=48)
    mat, md = _vq_material(case, 2, ntc.PREC_F16, 304)
    q = gen.random_queries(2 * 4096 + 3, md.mips, seed=4086)
    ntc.ntc_set_decode_warpgroups(nwg)
    try:
        out = to_np(ntc.ntc_decode(mat, torch.from_numpy(q).to(DEV)))
        tri = to_np(ntc.ntc_decode(mat, torch.from_numpy(q[:1000]).to(DEV),
                                   filter=ntc.FILTER_TRILINEAR))
    finally:
        ntc.ntc_set_decode_warpgroups(0)
    assert ntc.ntc_device_status() == ntc.OK
    assert np.abs(out - md.decode(q)).max() <= OUT_TOL
    assert np.abs(tri - md.decode_trilinear(q[:1000])).max() <= OUT_TOL


def test_vq_refusals():
    case = make_case(seed=88, width=256, height=256, channels=8, c0=8, c1=8, k_in=32)
    mat, _ = _vq_material(case, 2, ntc.PREC_F16, 301)
    q = torch.from_numpy(gen.random_queries(256, case.mips, seed=4088)).to(DEV)
    with pytest.raises(ntc.NTCError):
        ntc.ntc_decode(mat, q, flags=ntc.FLAG_NOISE)
    with pytest.raises(ntc.NTCError):
        ntc.Batch([mat], [256], ntc.FILTER_NEAREST)


# ------------------------------------------------------------- training ---
def _vq_trainer(case, cb, precision=ntc.PREC_F16, total=10, beta=0.25):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, w[0::2], w[1::2],
                       case.k_in, precision, case.act, case.out_act, total_steps=total,
                       codebook0=cb, vq_beta=beta)


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
def test_vq_training_step_gradients_match_oracle(precision):
    """One step of a vector-quantised G0 (GRAD_ONLY): the step's indices
    bit-exact against the oracle's assignment of the same latents; the
    gradients of the latents (the decoder's gradient at q, straight through,
    plus the commitment term), of the codebooks (codebook term), of G1 and of
    the MLP against the oracle (noise on G1 only)."""
    case = make_case(seed=89, width=256, height=256, channels=8, c0=8, c1=12, k_in=48)
    cb = _codebooks(2, 8, 302)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(256, 256, 8, seed=1089))
    tr = _vq_trainer(case, cb, precision)
    step, seed, batch = 2, 818, 9 * 128 + 21
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    idx, q, dz, dcb = oracle.vq_train_terms(case.val0, cb, 0.25)
    got_idx = tr.vq_idx.cpu().numpy()
    assert np.array_equal(got_idx, np.concatenate([i.reshape(-1) for i in idx]))
    w = [np.asarray(a, np.float64) for a in case.weights]
    if precision == ntc.PREC_F16:
        for i in range(0, len(w), 2):
            w[i] = case.weights[i].astype(np.float16).astype(np.float64)
    md = oracle.Model(case.width, case.height, 8, 8, 12, case.n0, case.n1, case.q0, case.q1, q,
                      [v.astype(np.float64) for v in case.val1], w, 48, vq_g0=True)
    xym = oracle.sample_batch(seed, step, batch, 256, 256, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    refs = [gq + d for gq, d in zip(g["grid0"], dz)] + g["grid1"] + g["w"] + [dcb]
    L = len(case.val0)
    check_grads(tr.grad_views[:-1], refs[:-1], 2 * L, precision == ntc.PREC_F16)
    assert rel_err(to_np(tr.grad_views[-1]), dcb) <= 1e-4   # codebooks: FP32 sums only


def test_vq_training_reduces_loss_and_exports():
    case = make_case(seed=90, width=128, height=128, channels=8, c0=8, c1=12, k_in=48)
    cb = _codebooks(2, 8, 303)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 8, seed=1090))
    tr = _vq_trainer(case, cb, total=300)
    target = ntc.Target(chain)
    first = ntc.ntc_train_step(tr, target, 4096, 13).item()
    for _ in range(298):
        ntc.ntc_train_step(tr, target, 4096, 13)
    last = ntc.ntc_train_step(tr, target, 4096, 13).item()
    assert ntc.ntc_device_status() == ntc.OK
    assert np.isfinite(last) and last < 0.5 * first, (first, last)
    m = tr.export(ntc.PREC_F16)
    assert m.struct.vq_books == 2 and m.grids0[0].dtype == torch.uint8
    cbn = tr.codebook.cpu().numpy()
    g0 = [oracle.vq_reconstruct(g.cpu().numpy(), cbn) for g in m.grids0]
    idx1 = [ntc.ntc_unpack(g.reshape(-1, g.shape[-1]), 12, 4, case.q1)[0].cpu().numpy()
            .reshape(g.shape[0], g.shape[1], 12) for g in m.grids1]
    w = []
    for wl, bl in zip(m.weights, m.biases):
        w += [to_np(wl), to_np(bl)]
    md = oracle.Model(128, 128, 8, 8, 12, 16, 16, case.q0, case.q1, g0,
                      [oracle.dequantize(i, 16, case.q1) for i in idx1], w, 48)
    q = gen.random_queries(3000, md.mips, seed=4090)
    out = to_np(ntc.ntc_decode(m, torch.from_numpy(q).to(DEV)))
    assert np.abs(out - md.decode(q)).max() <= OUT_TOL
