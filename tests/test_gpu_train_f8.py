"""The fused training step in the FP8-E4M3 form (R24: the paper trains with
half-precision tensor cores, Sec. 5.1, and leaves lower precision to future
work, Sec. 7): E4M3 forward on kind::f8f6f4 tensor cores with power-of-two
per-layer scales, FP16 backward on the same values, straight-through
reverse mode.  Against the oracle's FP8 form (Model.f8_form, pinned
separately): loss within 2e-3, every tensor's gradient within 1e-2, with
the scales the step used (read back from the trainer)."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import check_grads, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _trainer(case, sa, total=50):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                       [w[1], w[3], w[5]], case.k_in, ntc.PREC_F8, case.act, case.out_act,
                       total_steps=total, f8_act_scales=sa)


@pytest.mark.parametrize("act,out_act", [(0, 0), (1, 1)])
@pytest.mark.parametrize("shape", [
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=64),
    dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32),
    dict(width=256, height=128, channels=9, c0=12, c1=20, k_in=64),
])
def test_f8_train_gradients_match_fp8_oracle(shape, act, out_act):
    case = make_case(seed=141, act=act, out_act=out_act, **shape)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1141))
    sa = [1.0 / 256, 4.0 / 256, 4.0 / 256]
    tr = _trainer(case, sa)
    step, batch, seed = 2, 9 * 128 + 77, 919
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    sc = to_np(tr.f8_scale)
    s_w, s_a = list(sc[:3]), list(sc[3:6])
    assert s_a == sa  # no maxima recorded before this step: the initial scales
    for l in range(3):  # power-of-two weight scales with max|W| / s_w <= 448
        m = np.abs(case.weights[2 * l]).max()
        assert np.log2(s_w[l]) == np.round(np.log2(s_w[l])) and m / s_w[l] <= 448.0 < 2 * m / s_w[l]
    # the step recorded this step's layer-input maxima (for the next step's scales)
    assert np.all(sc[6:9] > 0)
    md = case.oracle_model(weights=[np.asarray(a, np.float64) for a in case.weights],
                           quantized=False).f8_form(s_w, s_a)
    xym = oracle.sample_batch(seed, step, batch, case.width, case.height, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(case.val0), True)


def test_f8_training_lowers_loss_and_updates_scales():
    """Full FP8 steps (pre-pass, noise, fused step, Adam): the loss falls like
    the FP16 step's, the activation scales follow the recorded maxima
    (powers of two), and the FP8 export decodes close to the FP16 export."""
    case = make_case(128, 128, 8, 8, 8, k_in=32, seed=142)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 8, seed=1142))
    target = ntc.Target(chain)
    curves = {}
    trs = {}
    for prec in (ntc.PREC_F16, ntc.PREC_F8):
        w = case.weights
        tr = ntc.Trainer(128, 128, 8, 8, 8, 4, 4, case.q0, case.q1, case.val0, case.val1,
                         [w[0], w[2], w[4]], [w[1], w[3], w[5]], 32, prec, total_steps=300,
                         f8_act_scales=[1.0 / 256, 1.0 / 64, 1.0 / 64] if prec == ntc.PREC_F8 else None)
        curves[prec] = [ntc.ntc_train_step(tr, target, 4096, 9).item() for _ in range(300)]
        trs[prec] = tr
    assert ntc.ntc_device_status() == ntc.OK
    a, b = np.mean(curves[ntc.PREC_F16][-20:]), np.mean(curves[ntc.PREC_F8][-20:])
    assert b < 0.5 * np.mean(curves[ntc.PREC_F8][:5])
    assert abs(a - b) <= 0.15 * a, (a, b)
    sa = to_np(trs[ntc.PREC_F8].f8_scale)[3:6]
    assert np.all(np.log2(sa) == np.round(np.log2(sa)))
    m8 = trs[ntc.PREC_F8].export(ntc.PREC_F8)
    m16 = trs[ntc.PREC_F8].export(ntc.PREC_F16)
    q = torch.from_numpy(gen.random_queries(4096, m16.mips, seed=7)).cuda()
    d8, d16 = to_np(ntc.ntc_decode(m8, q)), to_np(ntc.ntc_decode(m16, q))
    assert ntc.ntc_device_status() == ntc.OK
    assert np.abs(d8 - d16).mean() < 1e-2
