"""GPU parity of the training step's gradients (FP32 CUDA-core form and the
tcgen05 FP16 form) against the FP64 oracle, through ntc_train_step with
NTC_FLAG_GRAD_ONLY (sampler, noise, forward, loss, backward; no update).

The oracle sees the weights as the step's forward sees them (FP16 copies of
the masters for the tensor-core form).  Bars (`check_grads`): 1e-2 relative
error (L2 norm) per tensor for both forms; the loss within 2e-3 relative
(FP16 activations).
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _trainer(case, precision, total=100):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                       [w[1], w[3], w[5]], case.k_in, precision, case.act, case.out_act,
                       total_steps=total)


def _oracle_weights(case, precision):
    w = [np.asarray(a, np.float64) for a in case.weights]
    if precision == ntc.PREC_F16:
        for i in (0, 2, 4):
            w[i] = case.weights[i].astype(np.float16).astype(np.float64)
    return w


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
@pytest.mark.parametrize("shape", [
    dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32),
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48),
    dict(width=256, height=128, channels=16, c0=12, c1=12, k_in=48),
    dict(width=32, height=32, channels=3, c0=3, c1=5, k_in=32),
])
def test_train_gradients_match_oracle(shape, precision):
    case = make_case(seed=71, **shape)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1071))
    tr = _trainer(case, precision)
    target = ntc.Target(chain)
    batch, seed, step = 5 * 256 + 77, 4242, 3
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, target, batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    assert int(tr.step_t.item()) == step  # no update, no advance
    md = case.oracle_model(weights=_oracle_weights(case, precision), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, case.width, case.height, md.mips)
    lref, gref = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    L = len(case.val0)
    check_grads(tr.grad_views, gref["grid0"] + gref["grid1"] + gref["w"], 2 * L,
                precision == ntc.PREC_F16)


@pytest.mark.parametrize("act,out_act", [(1, 0), (1, 1), (0, 1)])
@pytest.mark.parametrize("shape", [
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48),
    dict(width=64, height=32, channels=5, c0=6, c1=5, k_in=32),
])
def test_train_f16_activations_match_oracle(shape, act, out_act):
    """hardGELU hidden layers (act'(Z) kept in FP16 for the backward) and the
    identity output on the tensor-core step, against the oracle."""
    case = make_case(seed=73, act=act, out_act=out_act, **shape)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1073))
    tr = _trainer(case, ntc.PREC_F16)
    target = ntc.Target(chain)
    batch, seed, step = 3 * 256 + 5, 4343, 1
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, target, batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_oracle_weights(case, ntc.PREC_F16), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, case.width, case.height, md.mips)
    lref, gref = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, gref["grid0"] + gref["grid1"] + gref["w"], 2 * len(case.val0), True)


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
@pytest.mark.parametrize("step", [2, 9])
def test_train_crops_gradients_match_oracle(precision, step):
    """The crop sampler in the fused step (NTC_FLAG_CROPS, Sec. 5.1): one
    mip, 256 x 256 windows, a ragged last crop; neighbouring texels share
    grid cells, so many atomics of a warp land on one address."""
    case = make_case(seed=74, width=512, height=256, channels=8, c0=8, c1=8, k_in=32)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(case.width, case.height, case.channels,
                                                       seed=1074))
    tr = _trainer(case, precision)
    target = ntc.Target(chain)
    batch, seed = 65536 + 4099, 4545
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, target, batch, seed,
                              flags=ntc.FLAG_GRAD_ONLY | ntc.FLAG_CROPS).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_oracle_weights(case, precision), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, case.width, case.height, md.mips, crops=True)
    lref, gref = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    refs = gref["grid0"] + gref["grid1"] + gref["w"]
    for k, (v, r) in enumerate(zip(tr.grad_views, refs)):
        if not np.any(r):
            assert not np.any(to_np(v)), k   # grids of other levels get nothing
    check_grads(tr.grad_views, refs, 2 * len(case.val0), precision == ntc.PREC_F16)


def test_train_f16_many_tiles_per_pipeline():
    """~300 K texels on the bench's training layout (three pipelines per CTA,
    several tiles each): gradients of every tensor against the oracle."""
    case = make_case(seed=75, width=512, height=512, channels=12, c0=16, c1=16, k_in=48)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(512, 512, 12, seed=1075))
    tr = _trainer(case, ntc.PREC_F16)
    batch, seed, step = 300_001, 4646, 2
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_oracle_weights(case, ntc.PREC_F16), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, 512, 512, md.mips)
    lref, gref = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, gref["grid0"] + gref["grid1"] + gref["w"], 2 * len(case.val0), True)


def test_train_f16_full_step_and_accumulation():
    """GRAD_ONLY twice then a regular step equals the sum of three batches'
    gradients applied once (gradient accumulation); the scratch gradient is
    left zeroed."""
    case = make_case(128, 128, 12, 16, 16, k_in=48, seed=72)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 12, seed=1072))
    target = ntc.Target(chain)
    tr = _trainer(case, ntc.PREC_F16)
    ntc.ntc_train_step(tr, target, 1000, 5, flags=ntc.FLAG_GRAD_ONLY)
    g1 = tr.grad.clone()
    ntc.ntc_train_step(tr, target, 1000, 5, flags=ntc.FLAG_GRAD_ONLY)
    assert rel_err(to_np(tr.grad), 2 * to_np(g1)) < 1e-3
    p0 = tr.params.clone()
    ntc.ntc_train_step(tr, target, 1000, 5)
    assert ntc.ntc_device_status() == ntc.OK
    assert int(tr.step_t.item()) == 1
    assert float(tr.grad.abs().max()) == 0.0
    assert float((tr.params - p0).abs().max()) > 0
    # the FP16 weight copies follow the masters
    for wc, wm in zip(tr.material.weights, tr.w_master):
        assert torch.equal(wc, wm.half())


def test_train_f16_reduces_loss_like_fp32():
    """Both forms lower the loss on the same material at a similar rate."""
    case = make_case(128, 128, 8, 8, 8, k_in=32, seed=73)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 8, seed=1073))
    target = ntc.Target(chain)
    curves = {}
    for prec in (ntc.PREC_F32, ntc.PREC_F16):
        tr = _trainer(case, prec, total=300)
        curves[prec] = [ntc.ntc_train_step(tr, target, 4096, 9).item() for _ in range(300)]
    a, b = np.mean(curves[ntc.PREC_F32][-20:]), np.mean(curves[ntc.PREC_F16][-20:])
    assert a < 0.5 * np.mean(curves[ntc.PREC_F32][:5])
    assert abs(a - b) <= 0.1 * a, (a, b)


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
def test_dense_noise_pass_equals_noise_per_tap(precision):
    """The step with the trainer's noisy scratch (one dense noise pass, then
    gathers of noisy values) and without it (noise added per tap) see the
    same noisy grids: equal loss and gradients up to the order of the
    atomic sums."""
    case = make_case(256, 128, 12, 12, 12, k_in=48, seed=73)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(256, 128, 12, seed=1073))
    target = ntc.Target(chain)
    w = case.weights
    grads, losses = [], []
    for scratch in (True, False):
        tr = ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                         case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                         [w[1], w[3], w[5]], case.k_in, precision, total_steps=50,
                         noisy_scratch=scratch)
        tr.step_t.fill_(5)
        ntc.ntc_train_step(tr, target, 3 * 1024 + 5, 99, flags=ntc.FLAG_GRAD_ONLY)
        torch.cuda.synchronize()
        assert ntc.ntc_device_status() == ntc.OK
        grads.append(to_np(tr.grad))
        losses.append(tr.loss.item())
    assert abs(losses[0] - losses[1]) <= 1e-6 * abs(losses[1])
    assert rel_err(grads[0], grads[1]) < 1e-5



def test_fused_step_checks_a_stale_tag_itself():
    """After a regular step with seed s the library expects the next step
    with s to find the noisy copy current, and lets the fused kernel check
    the tag instead of launching the noise pass.  Moving the step counter by
    hand makes the tag stale: the fused step must then add the noise per tap,
    so its loss and gradient equal those of a trainer without the noisy
    scratch in the same state."""
    case = make_case(128, 64, 12, 12, 12, k_in=48, seed=77)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 64, 12, seed=1077))
    target = ntc.Target(chain)
    w = case.weights
    a = _trainer(case, ntc.PREC_F16, total=40)
    b = ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                    case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                    [w[1], w[3], w[5]], case.k_in, ntc.PREC_F16, case.act, case.out_act,
                    total_steps=40, noisy_scratch=False)
    for tr in (a, b):
        ntc.ntc_train_step(tr, target, 2048 + 17, 9)   # a: Adam writes the copy of step 1
    torch.cuda.synchronize()
    assert a.noisy_tag.cpu().tolist() == [9, 1]
    losses, grads = [], []
    for tr in (a, b):
        tr.step_t.fill_(5)                             # a's tag {9, 1} is now stale
        ntc.ntc_train_step(tr, target, 2048 + 17, 9, flags=ntc.FLAG_GRAD_ONLY)
        torch.cuda.synchronize()
        assert ntc.ntc_device_status() == ntc.OK
        losses.append(tr.loss.item())
        grads.append(to_np(tr.grad))
    # the first step's parameters differ by the order of its atomic sums
    assert abs(losses[0] - losses[1]) <= 1e-5 * abs(losses[1])
    assert rel_err(grads[0], grads[1]) < 1e-4

def _expected_noisy(tr, case, seed, step):
    """params + the oracle's noise of (seed, step) for every grid value, summed
    in FP32 (the dense noise pass's arithmetic), per grid view."""
    out = []
    for k, views in ((0, tr.material.grids0), (1, tr.material.grids1)):
        c, q = (case.c1, case.q1) if k else (case.c0, case.q0)
        for j, v in enumerate(views):
            p = v.detach().cpu().numpy().reshape(-1, c).astype(np.float32)
            noise = np.array([[oracle.noise_value(seed, step, j, k, cell, ch, c, q)
                               for ch in range(c)] for cell in range(p.shape[0])], np.float32)
            out.append((p + noise).reshape(-1))
    return out


def _noisy_views(tr):
    base = tr.params.data_ptr()
    res = []
    for views in (tr.material.grids0, tr.material.grids1):
        for v in views:
            off = (v.data_ptr() - base) // 4
            res.append(tr.noisy[off:off + v.numel()].cpu().numpy())
    return res


def test_noise_folded_into_adam_matches_the_noise_pass():
    """With noisy_tag each step's Adam writes the next step's noisy grids and
    the next noise pass skips.  The copy Adam writes equals params + the
    oracle's noise of (seed, next step) bit for bit; with changing seeds and
    a NO_NOISE step in between, every step's loss equals that of a trainer
    that runs the dense noise pass every step."""
    case = make_case(128, 64, 12, 12, 12, k_in=48, seed=76)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 64, 12, seed=1076))
    target = ntc.Target(chain)
    a, b = _trainer(case, ntc.PREC_F16, total=40), _trainer(case, ntc.PREC_F16, total=40)
    b.noisy_tag = None  # the noise pass every step
    plan = [(5, 0), (5, 0), (6, 0), (6, ntc.FLAG_NO_NOISE), (6, 0), (6, 0)]
    for i, (seed, flags) in enumerate(plan):
        la = ntc.ntc_train_step(a, target, 2048 + 17, seed, flags=flags).item()
        lb = ntc.ntc_train_step(b, target, 2048 + 17, seed, flags=flags).item()
        assert abs(la - lb) <= 1e-5 * lb, (seed, flags, la, lb)
        if not flags:
            torch.cuda.synchronize()
            for got, want in zip(_noisy_views(a), _expected_noisy(a, case, seed, i + 1)):
                assert np.array_equal(got, want), i
    assert ntc.ntc_device_status() == ntc.OK
    assert a.noisy_tag.cpu().tolist() == [6, len(plan)]
    assert rel_err(to_np(a.params), to_np(b.params)) <= 1e-3
