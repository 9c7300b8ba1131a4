"""Three hidden layers (Sec. 4.4 gives activations to three layers after the first;
the network sizes of Table 5): K -> 64 -> 64 -> 64 -> C.  Parity with the
FP64 oracle of the same model: FP32 and FP16 (warp-specialised) decode with
every filter, FP16 tensor-core training gradients (bilinear ReLU, and the
paper's decoder form: learned G0, hardGELU, identity output), and the calls
that refuse this depth."""
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
    dict(width=512, height=512, channels=16, c0=12, c1=12, k_in=48),              # fast layout
    dict(width=256, height=128, channels=5, c0=6, c1=5, bits0=2, bits1=8, k_in=32, act=1),
    dict(width=256, height=256, channels=9, c0=16, c1=12, k_in=96, act=1, out_act=1,
         interp0=1),                                                               # paper form
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


def _decode(mat, q, **kw):
    out = ntc.ntc_decode(mat, _uvl(q), **kw)
    assert ntc.ntc_device_status() == ntc.OK
    return to_np(out)


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
@pytest.mark.parametrize("shape", SHAPES)
def test_decode_three_hidden_layers_matches_oracle(shape, precision):
    case = make_case(seed=81, hidden_layers=3, **shape)
    mat, md = device_material(case, precision=precision)
    assert md.hidden_layers == 3 and mat.struct.hidden_layers == 3
    q = gen.random_queries(3 * 4096 + 19, md.mips, seed=4081)
    assert np.abs(_decode(mat, q) - md.decode(q)).max() <= OUT_TOL
    tri = _decode(mat, q[:1500], filter=ntc.FILTER_TRILINEAR)
    assert np.abs(tri - md.decode_trilinear(q[:1500])).max() <= OUT_TOL
    st = _decode(mat, q[:1500], filter=ntc.FILTER_STOCHASTIC, noise_seed=3, noise_step=7)
    assert np.abs(st - md.decode_stochastic(q[:1500], 3, 7)).max() <= OUT_TOL


def test_every_launch_shape_runs_three_hidden_layers():
    """Shapes 2-4 route a three-hidden-layer material to the warp-specialised
    kernel: the same outputs whatever the setting."""
    case = make_case(seed=82, hidden_layers=3, **SHAPES[0])
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = gen.random_queries(5000, md.mips, seed=4082)
    ref = md.decode(q)
    for nwg in (2, 3, 4, 5):
        ntc.ntc_set_decode_warpgroups(nwg)
        try:
            assert np.abs(_decode(mat, q) - ref).max() <= OUT_TOL, nwg
        finally:
            ntc.ntc_set_decode_warpgroups(0)


def _trainer(case, total=10):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, w[0::2], w[1::2],
                       case.k_in, ntc.PREC_F16, case.act, case.out_act, total_steps=total,
                       interp0=case.interp0)


def _f16_oracle_weights(case):
    w = [np.asarray(a, np.float64) for a in case.weights]
    for i in range(0, len(w), 2):
        w[i] = case.weights[i].astype(np.float16).astype(np.float64)
    return w


@pytest.mark.parametrize("batch", [5 * 128 + 33, 150_000])
@pytest.mark.parametrize("shape", [
    dict(width=256, height=256, channels=12, c0=16, c1=16, k_in=48),
    dict(width=256, height=256, channels=9, c0=16, c1=12, k_in=96, act=1, out_act=1, interp0=1),
])
def test_train_three_hidden_layers_gradients_match_oracle(shape, batch):
    """FP16 tensor-core step through the third hidden layer: loss and every
    tensor's gradient (grids, W1..W3, Wh and their biases) against the
    oracle's reverse mode, noise on; the large batch gives every pipeline
    several tiles."""
    case = make_case(seed=83, hidden_layers=3, **shape)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1083))
    tr = _trainer(case)
    step, seed = 3, 919
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_f16_oracle_weights(case), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, case.width, case.height, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    assert len(tr.grad_views) == 2 * len(md.grids0) + 8
    check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(md.grids0), True)


def test_train_three_hidden_layers_reduces_loss_and_exports():
    """Full steps of the paper's decoder form with three hidden layers lower
    the loss; the export decodes like the oracle of the exported model."""
    case = make_case(128, 128, 9, 12, 10, k_in=80, act=1, out_act=1, seed=84, interp0=1,
                     hidden_layers=3)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 9, seed=1084))
    tr = _trainer(case, total=300)
    target = ntc.Target(chain)
    first = ntc.ntc_train_step(tr, target, 4096, 12).item()
    for _ in range(298):
        ntc.ntc_train_step(tr, target, 4096, 12)
    last = ntc.ntc_train_step(tr, target, 4096, 12).item()
    assert ntc.ntc_device_status() == ntc.OK
    assert np.isfinite(last) and last < 0.5 * first, (first, last)
    m = tr.export(ntc.PREC_F16)
    assert len(m.weights) == 4 and m.struct.hidden_layers == 3
    idx0 = [ntc.ntc_unpack(g.reshape(-1, g.shape[-1]), 12, 4, case.q0)[0].cpu().numpy()
            .reshape(g.shape[0], g.shape[1], 12) for g in m.grids0]
    idx1 = [ntc.ntc_unpack(g.reshape(-1, g.shape[-1]), 10, 4, case.q1)[0].cpu().numpy()
            .reshape(g.shape[0], g.shape[1], 10) for g in m.grids1]
    w = []
    for wl, bl in zip(m.weights, m.biases):
        w += [to_np(wl), to_np(bl)]
    md = oracle.Model(128, 128, 9, 12, 10, 16, 16, case.q0, case.q1,
                      [oracle.dequantize(i, 16, case.q0) for i in idx0],
                      [oracle.dequantize(i, 16, case.q1) for i in idx1], w, 80, act=1, out_act=1,
                      interp0=1)
    q = gen.random_queries(3000, md.mips, seed=4084)
    assert np.abs(_decode(m, q) - md.decode(q)).max() <= OUT_TOL


def test_three_hidden_layers_refusals():
    case = make_case(seed=85, hidden_layers=3, **SHAPES[0])
    m32, _ = device_material(case, precision=ntc.PREC_F32, packed=False)
    q = _uvl(gen.random_queries(256, case.mips, seed=4085))
    # the FP32 reverse mode and FP32 training hold two hidden layers
    with pytest.raises(ntc.NTCError):
        ntc.ntc_backward(m32, q, torch.zeros((256, 16), device=DEV), ntc.grads_struct(m32))
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, 16, seed=1085))
    w = case.weights
    tr = ntc.Trainer(case.width, case.height, 16, 12, 12, 4, 4, case.q0, case.q1, case.val0,
                     case.val1, w[0::2], w[1::2], 48, ntc.PREC_F32, total_steps=10)
    with pytest.raises(ntc.NTCError):
        ntc.ntc_train_step(tr, ntc.Target(chain), 256, 1)
    # batches decode two hidden layers
    m16, _ = device_material(case, precision=ntc.PREC_F16)
    with pytest.raises(ntc.NTCError):
        ntc.Batch([m16], [256], ntc.FILTER_NEAREST)
