"""Many materials' optimisation steps in one persistent launch
(ntc_train_step_batched) against the FP64 oracle and against one
ntc_train_step per material.

Six materials of different sides, channel counts, feature widths and input
widths, with batches that include 0 (the material sits out) and 1 (one
valid row in a tile).  Gradients per tensor within 1e-2 of the oracle's
reverse mode (the same bar as the single-material step), and within 1e-5 of
the single-material step's (the same arithmetic, up to the order of the
atomic sums).
"""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import check_grads, rel_err, to_np

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32),
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48),
    dict(width=256, height=128, channels=16, c0=12, c1=12, k_in=48),
    dict(width=32, height=32, channels=3, c0=3, c1=5, k_in=32),
    dict(width=128, height=64, channels=8, c0=8, c1=12, k_in=48),
    dict(width=64, height=64, channels=16, c0=16, c1=8, k_in=48),
]
BATCHES = [1357, 0, 3000, 1, 700, 129]
SEED = 9090


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _setup(k, act=0, out_act=0):
    case = make_case(seed=80 + k, act=act, out_act=out_act, **SHAPES[k])
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1080 + k))
    w = case.weights
    tr = ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                     case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                     [w[1], w[3], w[5]], case.k_in, ntc.PREC_F16, act, out_act, total_steps=50)
    return case, chain, tr, ntc.Target(chain)


def _oracle_weights(case):
    w = [np.asarray(a, np.float64) for a in case.weights]
    for i in (0, 2, 4):
        w[i] = case.weights[i].astype(np.float16).astype(np.float64)
    return w


@pytest.mark.parametrize("act,out_act", [(0, 0), (1, 1)])
def test_batched_gradients_match_oracle_and_single_steps(act, out_act):
    sets = [_setup(k, act, out_act) for k in range(len(SHAPES))]
    for k, (_, _, tr, _) in enumerate(sets):
        tr.step_t.fill_(k)  # a different step (noise, samples) per material
    tb = ntc.TrainBatch([s[2] for s in sets], [s[3] for s in sets], BATCHES, SEED,
                        flags=ntc.FLAG_GRAD_ONLY)
    loss = ntc.ntc_train_step_batched(tb).cpu().numpy()
    assert ntc.ntc_device_status() == ntc.OK
    for k, (case, chain, tr, target) in enumerate(sets):
        assert int(tr.step_t.item()) == k  # gradient only: no update, no advance
        if BATCHES[k] == 0:
            assert loss[k] == 0.0
            assert float(tr.grad.abs().max()) == 0.0
            continue
        md = case.oracle_model(weights=_oracle_weights(case), quantized=False)
        xym = oracle.sample_batch(SEED + k, k, BATCHES[k], case.width, case.height, md.mips)
        lref, gref = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(SEED + k, k))
        assert abs(loss[k] - lref) <= 2e-3 * lref, (k, loss[k], lref)
        refs = gref["grid0"] + gref["grid1"] + gref["w"]
        if BATCHES[k] > 1:
            check_grads(tr.grad_views, refs, 2 * len(case.val0), True)
        else:
            # one texel: a tensor's gradient is one texel's, often ~0 at the
            # level it does not touch -- compare the whole gradient
            got = np.concatenate([to_np(v).reshape(-1) for v in tr.grad_views])
            assert rel_err(got, np.concatenate([r.reshape(-1) for r in refs])) <= 1e-2
        # the same step through the single-material entry point
        g_batched = to_np(tr.grad)
        tr.grad.zero_()
        l1 = ntc.ntc_train_step(tr, target, BATCHES[k], SEED + k, flags=ntc.FLAG_GRAD_ONLY).item()
        assert abs(l1 - loss[k]) <= 1e-5 * l1, (k, l1, loss[k])
        assert rel_err(g_batched, to_np(tr.grad)) <= 1e-5, k


def test_batched_full_steps_equal_single_steps_and_replay_in_a_graph():
    """Three batched steps (Adam included; its last block advances the step
    counters) equal three single-material steps per material; the same
    batched step captured in a CUDA graph and replayed continues identically."""
    a = [_setup(k) for k in range(len(SHAPES))]
    b = [_setup(k) for k in range(len(SHAPES))]
    tb = ntc.TrainBatch([s[2] for s in a], [s[3] for s in a], BATCHES, SEED)
    for step in range(3):
        la = ntc.ntc_train_step_batched(tb).cpu().numpy()
        for k, (_, _, tr, tg) in enumerate(b):
            if BATCHES[k]:
                lb = ntc.ntc_train_step(tr, tg, BATCHES[k], SEED + k).item()
                assert abs(la[k] - lb) <= 1e-4 * lb, (step, k, la[k], lb)
    assert ntc.ntc_device_status() == ntc.OK
    for k in range(len(SHAPES)):
        ta, tbk = a[k][2], b[k][2]
        want = 3 if BATCHES[k] else 0
        assert int(ta.step_t.item()) == int(tbk.step_t.item()) == want, k
        assert float(ta.grad.abs().max()) == 0.0
        if BATCHES[k]:
            assert rel_err(to_np(ta.params), to_np(tbk.params)) <= 1e-4, k
            for wc, wm in zip(ta.material.weights, ta.w_master):
                assert torch.equal(wc, wm.half())
    # graph capture of the batched step, replayed twice, against eager steps
    # of the second copy
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ntc.ntc_train_step_batched(tb, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        g.replay()
        torch.cuda.synchronize()
        for k, (_, _, tr, tg) in enumerate(b):
            if BATCHES[k]:
                ntc.ntc_train_step(tr, tg, BATCHES[k], SEED + k)
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    for k in range(len(SHAPES)):
        assert int(a[k][2].step_t.item()) == int(b[k][2].step_t.item())
        if BATCHES[k]:
            assert rel_err(to_np(a[k][2].params), to_np(b[k][2].params)) <= 1e-4, k


@pytest.mark.parametrize("variant", ["learned", "three_hidden", "crops"])
def test_batched_variants_equal_single_steps(variant):
    """The paper's decoder form (learned G0, hardGELU, identity), three hidden
    layers and crop batches in the batched step: each material's loss and
    gradient equal its single-material step's (same arithmetic, atomic order
    aside); the learned form also against the oracle."""
    flags = ntc.FLAG_GRAD_ONLY | (ntc.FLAG_CROPS if variant == "crops" else 0)
    shapes = [dict(width=128, height=128, channels=9, c0=12, c1=10, k_in=80),
              dict(width=256, height=128, channels=6, c0=8, c1=12, k_in=64),
              dict(width=64, height=64, channels=12, c0=16, c1=12, k_in=96)]
    kw = dict(act=1, out_act=1, interp0=1) if variant == "learned" else {}
    if variant == "three_hidden":
        kw = dict(hidden_layers=3)
    if variant == "crops":
        shapes = [dict(width=512, height=256, channels=8, c0=8, c1=8, k_in=32),
                  dict(width=256, height=256, channels=12, c0=12, c1=12, k_in=48)]
    batches = [3000, 70000, 1] if variant != "crops" else [65536 + 4099, 70000]
    sets = []
    for k, shape in enumerate(shapes):
        case = make_case(seed=160 + k, **kw, **shape)
        chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height,
                                                           case.channels, seed=1160 + k))
        w = case.weights
        tr = ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                         case.bits1, case.q0, case.q1, case.val0, case.val1, w[0::2], w[1::2],
                         case.k_in, ntc.PREC_F16, case.act, case.out_act, total_steps=20,
                         interp0=case.interp0)
        tr.step_t.fill_(k + 1)
        sets.append((case, chain, tr, ntc.Target(chain)))
    tb = ntc.TrainBatch([s[2] for s in sets], [s[3] for s in sets], batches, SEED, flags=flags)
    loss = ntc.ntc_train_step_batched(tb).cpu().numpy()
    assert ntc.ntc_device_status() == ntc.OK
    for k, (case, chain, tr, target) in enumerate(sets):
        g_batched = to_np(tr.grad)
        tr.grad.zero_()
        l1 = ntc.ntc_train_step(tr, target, batches[k], SEED + k, flags=flags).item()
        assert abs(l1 - loss[k]) <= 1e-5 * max(l1, 1e-12), (variant, k, l1, loss[k])
        assert rel_err(g_batched, to_np(tr.grad)) <= 1e-5, (variant, k)
        if variant == "learned" and batches[k] > 1:
            w16 = [np.asarray(a, np.float64) for a in case.weights]
            for i in range(0, len(w16), 2):
                w16[i] = case.weights[i].astype(np.float16).astype(np.float64)
            md = case.oracle_model(weights=w16, quantized=False)
            xym = oracle.sample_batch(SEED + k, k + 1, batches[k], case.width, case.height, md.mips)
            lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym),
                                       noise=(SEED + k, k + 1))
            assert abs(l1 - lref) <= 2e-3 * lref
            check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(case.val0), True)
