"""Grids of 17-20 features per cell (the paper's profile 0.5 stores a
20-channel G1, the NTC profiles table in Sec. 6): 4-bit cells of 16 bytes,
three groups of eight inputs per grid.  Decode (FP32 and FP16 forms,
nearest and trilinear, batched) and the FP16 tensor-core training step
(gradients of every tensor within 1e-2 of the oracle; dX goes through the
shared-memory staging rows) with bilinear G0, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, check_grads, device_material, to_np

pytestmark = pytest.mark.gpu
OUT_TOL = 2e-3

SHAPES = [
    dict(width=256, height=256, channels=9, c0=12, c1=20, k_in=48),   # profile 0.5, bilinear G0
    dict(width=128, height=256, channels=12, c0=20, c1=12, k_in=48),  # a wide G0
    dict(width=128, height=128, channels=16, c0=17, c1=3, k_in=48),   # odd widths
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
@pytest.mark.parametrize("shape", SHAPES)
def test_wide_grid_decode_matches_oracle(shape, precision):
    case = make_case(seed=131, **shape)
    mat, md = device_material(case, precision=precision)
    q = gen.random_queries(5 * 128 + 19, md.mips, seed=4131)
    tol = 2e-5 if precision == ntc.PREC_F32 else OUT_TOL
    for filt, ref in ((ntc.FILTER_NEAREST, md.decode(q)),
                      (ntc.FILTER_TRILINEAR, md.decode_trilinear(q[:1500]))):
        got = to_np(ntc.ntc_decode(mat, _uvl(q if filt == ntc.FILTER_NEAREST else q[:1500]),
                                   filter=filt))
        assert ntc.ntc_device_status() == ntc.OK
        assert np.abs(got - ref).max() <= tol, filt


def test_wide_grid_batched_decode_matches_oracle():
    a = make_case(seed=132, **SHAPES[0])
    b = make_case(128, 128, 8, 12, 12, k_in=48, seed=133)
    mats = [device_material(a, precision=ntc.PREC_F16), device_material(b, precision=ntc.PREC_F16)]
    qs = [gen.random_queries(901, mats[0][1].mips, seed=4132),
          gen.random_queries(333, mats[1][1].mips, seed=4133)]
    batch = ntc.Batch([m for m, _ in mats], [len(q) for q in qs])
    out = to_np(ntc.ntc_decode_batched(batch, _uvl(np.concatenate(qs))))
    assert ntc.ntc_device_status() == ntc.OK
    for i, ((m, md), q) in enumerate(zip(mats, qs)):
        got = out[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(q), m.channels)
        assert np.abs(got - md.decode(q)).max() <= OUT_TOL, i


@pytest.mark.parametrize("shape", SHAPES)
def test_wide_grid_f16_training_gradients_match_oracle(shape):
    case = make_case(seed=134, **shape)
    w, h, c = case.width, case.height, case.channels
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(w, h, c, seed=1134))
    wt = case.weights
    tr = ntc.Trainer(w, h, c, case.c0, case.c1, case.bits0, case.bits1, case.q0, case.q1,
                     case.val0, case.val1, [wt[0], wt[2], wt[4]], [wt[1], wt[3], wt[5]],
                     case.k_in, ntc.PREC_F16, total_steps=10)
    step, batch, seed = 3, 9 * 128 + 7, 818
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    w16 = [np.asarray(a, np.float64) for a in wt]
    for i in (0, 2, 4):
        w16[i] = wt[i].astype(np.float16).astype(np.float64)
    md = case.oracle_model(weights=w16, quantized=False)
    xym = oracle.sample_batch(seed, step, batch, w, h, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(md.grids0), True)
