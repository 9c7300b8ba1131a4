"""Learned interpolation of G0 (Sec. 4.3.1): the four G0 taps concatenated in
the MLP input (the paper's decoder input, 4 c0 + c1 + 13 values) with the
paper's hardGELU and identity output.  Parity with the FP64 oracle of the
same model: FP32 form (decode and gradients), FP16 tensor-core decode
(nearest, trilinear, stochastic; warp-specialised and batched launches) and
FP16 tensor-core training (gradients of every tensor)."""
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

# (c0 x b0, c1 x b1) of the paper's four profiles (the NTC profiles table,
# Sec. 6), at small sides
PROFILES = [
    dict(width=256, height=256, channels=9, c0=8, c1=12, bits0=2, bits1=4, k_in=64),   # 0.2
    dict(width=256, height=128, channels=9, c0=12, c1=20, bits0=4, bits1=4, k_in=96),  # 0.5
    dict(width=128, height=128, channels=9, c0=12, c1=10, bits0=2, bits1=4, k_in=80),  # 1.0
    dict(width=256, height=256, channels=9, c0=16, c1=12, bits0=4, bits1=4, k_in=96),  # 2.25
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


def _queries(md, n, seed):
    rng = np.random.default_rng(seed)
    q = np.empty((n, 3), np.float32)
    q[:, :2] = rng.random((n, 2))
    q[:, 2] = rng.uniform(-0.5, md.mips + 0.5, n)
    return q


@pytest.mark.parametrize("shape", PROFILES)
def test_learned_decode_fp32_matches_oracle(shape):
    case = make_case(seed=91, act=1, out_act=1, interp0=1, **shape)
    mat, md = device_material(case)
    q = _queries(md, 1500, 4091)
    for filt, ref in ((ntc.FILTER_NEAREST, md.decode(q)), (ntc.FILTER_TRILINEAR, md.decode_trilinear(q)),
                      (ntc.FILTER_STOCHASTIC, md.decode_stochastic(q, 4, 2))):
        got = to_np(ntc.ntc_decode(mat, _uvl(q), filter=filt, noise_seed=4, noise_step=2))
        assert np.abs(got - ref).max() < 2e-5, filt


@pytest.mark.parametrize("shape", PROFILES)
def test_learned_decode_f16_matches_oracle(shape):
    case = make_case(seed=92, act=1, out_act=1, interp0=1, **shape)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = _queries(md, 7 * 128 + 41, 4092)
    for nwg in (0, 4):  # shape 4 routes K > 48 to the warp-specialised kernel too
        ntc.ntc_set_decode_warpgroups(nwg)
        try:
            for filt, ref in ((ntc.FILTER_NEAREST, md.decode(q)),
                              (ntc.FILTER_TRILINEAR, md.decode_trilinear(q))):
                got = to_np(ntc.ntc_decode(mat, _uvl(q), filter=filt))
                assert ntc.ntc_device_status() == ntc.OK
                assert np.abs(got - ref).max() <= OUT_TOL, (nwg, filt)
        finally:
            ntc.ntc_set_decode_warpgroups(0)


def test_learned_and_bilinear_in_one_batch():
    # profile 2.25's fast layout (profile 0.5's 20-channel G1 decodes on the
    # generic layout, whose K = 96 plan does not fit the batched kernel's
    # four per-warpgroup material regions: refused, see below)
    a = make_case(seed=93, act=1, out_act=1, interp0=1, **PROFILES[3])
    b = make_case(128, 128, 8, 12, 12, k_in=48, seed=94)
    mats = [device_material(a, precision=ntc.PREC_F16), device_material(b, precision=ntc.PREC_F16)]
    qs = [_queries(mats[0][1], 777, 4093), _queries(mats[1][1], 555, 4094)]
    batch = ntc.Batch([m for m, _ in mats], [len(q) for q in qs])
    out = to_np(ntc.ntc_decode_batched(batch, _uvl(np.concatenate(qs))))
    assert ntc.ntc_device_status() == ntc.OK
    for i, ((m, md), q) in enumerate(zip(mats, qs)):
        got = out[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(q), m.channels)
        assert np.abs(got - md.decode(q)).max() <= OUT_TOL, i


def test_learned_gradients_fp32_match_oracle():
    """FP32 fused step with learned interpolation (K <= 64): gradients of
    every tensor against the oracle's reverse mode, noise on."""
    case = make_case(64, 64, 5, 8, 4, k_in=64, act=1, out_act=1, seed=95, interp0=1)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(64, 64, 5, seed=1095))
    w = case.weights
    tr = ntc.Trainer(64, 64, 5, 8, 4, 4, 4, case.q0, case.q1, case.val0, case.val1,
                     [w[0], w[2], w[4]], [w[1], w[3], w[5]], 64, ntc.PREC_F32, act=1, out_act=1,
                     total_steps=10)
    tr.material.interp0 = 1
    tr.step_t.fill_(2)
    target = ntc.Target(chain)
    batch, seed = 3 * 128 + 9, 515
    ntc.ntc_train_step(tr, target, batch, seed, flags=ntc.FLAG_GRAD_ONLY | ntc.FLAG_SIMT)
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(quantized=False)
    xym = oracle.sample_batch(seed, 2, batch, 64, 64, md.mips)
    t = oracle.targets_of_xym(chain, xym)
    _, g = md.loss_grad_xym(xym, t, noise=(seed, 2))
    for got, ref in zip(tr.grad_views[:len(md.grids0)], g["grid0"]):
        assert rel_err(to_np(got), ref) < 1e-2
    for got, ref in zip(tr.grad_views[2 * len(md.grids0)::2], g["w"][0::2]):
        assert rel_err(to_np(got), ref) < 1e-2


def _f16_weights(case):
    w = [np.asarray(a, np.float64) for a in case.weights]
    for i in (0, 2, 4):
        w[i] = case.weights[i].astype(np.float16).astype(np.float64)
    return w


@pytest.mark.parametrize("dense_noise", [True, False])
@pytest.mark.parametrize("shape", PROFILES)
def test_learned_gradients_f16_tensor_cores_match_oracle(shape, dense_noise):
    """FP16 tcgen05 fused step of the paper-form decoder (learned G0,
    hardGELU, identity output) on the four profiles' layouts: loss and the
    gradient of every tensor against the oracle's reverse mode, noise on
    (dense noise pass, or noise added per tap)."""
    case = make_case(**shape, act=1, out_act=1, seed=97, interp0=1)
    w, h, c = case.width, case.height, case.channels
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(w, h, c, seed=1097))
    wt = case.weights
    tr = ntc.Trainer(w, h, c, case.c0, case.c1, case.bits0, case.bits1, case.q0, case.q1,
                     case.val0, case.val1, [wt[0], wt[2], wt[4]], [wt[1], wt[3], wt[5]],
                     case.k_in, ntc.PREC_F16, act=1, out_act=1, total_steps=10,
                     noisy_scratch=dense_noise, interp0=ntc.INTERP_LEARNED)
    step = 4
    tr.step_t.fill_(step)
    target = ntc.Target(chain)
    batch, seed = 7 * 128 + 33, 616
    loss = ntc.ntc_train_step(tr, target, batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_f16_weights(case), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, w, h, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(md.grids0), True)


@pytest.mark.parametrize("act,out_act", [(1, 1), (0, 0)])
def test_learned_gradients_f16_many_tiles_per_pipeline(act, out_act):
    """A batch of ~120 K texels: every pipeline of every CTA runs several
    tiles, so state kept across tiles (constant tiles, the shared
    weight-gradient accumulators) is exercised; profile 2.25's layout."""
    case = make_case(256, 256, 9, 16, 12, 4, 4, k_in=96, act=act, out_act=out_act, seed=99,
                     interp0=1)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(256, 256, 9, seed=1099))
    wt = case.weights
    tr = ntc.Trainer(256, 256, 9, 16, 12, 4, 4, case.q0, case.q1, case.val0, case.val1,
                     [wt[0], wt[2], wt[4]], [wt[1], wt[3], wt[5]], 96, ntc.PREC_F16, act=act,
                     out_act=out_act, total_steps=10, interp0=ntc.INTERP_LEARNED)
    step, batch, seed = 1, 120_000, 717
    tr.step_t.fill_(step)
    loss = ntc.ntc_train_step(tr, ntc.Target(chain), batch, seed, flags=ntc.FLAG_GRAD_ONLY).item()
    assert ntc.ntc_device_status() == ntc.OK
    md = case.oracle_model(weights=_f16_weights(case), quantized=False)
    xym = oracle.sample_batch(seed, step, batch, 256, 256, md.mips)
    lref, g = md.loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, step))
    assert abs(loss - lref) <= 2e-3 * lref, (loss, lref)
    check_grads(tr.grad_views, g["grid0"] + g["grid1"] + g["w"], 2 * len(md.grids0), True)


def test_learned_f16_training_reduces_loss():
    """A few hundred full FP16 steps of the paper-form decoder lower the loss
    and export a material whose packed decode follows the trained model."""
    case = make_case(128, 128, 9, 12, 10, 4, 4, k_in=80, act=1, out_act=1, seed=98, interp0=1)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 9, seed=1098))
    wt = case.weights
    tr = ntc.Trainer(128, 128, 9, 12, 10, 4, 4, case.q0, case.q1, case.val0, case.val1,
                     [wt[0], wt[2], wt[4]], [wt[1], wt[3], wt[5]], 80, ntc.PREC_F16, act=1,
                     out_act=1, total_steps=300, interp0=ntc.INTERP_LEARNED)
    target = ntc.Target(chain)
    first = ntc.ntc_train_step(tr, target, 4096, 11).item()
    for _ in range(298):
        ntc.ntc_train_step(tr, target, 4096, 11)
    last = ntc.ntc_train_step(tr, target, 4096, 11).item()
    assert ntc.ntc_device_status() == ntc.OK
    assert np.isfinite(last) and last < 0.5 * first, (first, last)
    m = tr.export(ntc.PREC_F16)
    assert m.interp0 == ntc.INTERP_LEARNED
    q = _queries(case.oracle_model(), 2048, 5)
    out = to_np(ntc.ntc_decode(m, _uvl(q)))
    assert np.isfinite(out).all()


def test_learned_fp32_training_beyond_k64_is_refused():
    case = make_case(64, 64, 5, 12, 4, k_in=80, seed=96, interp0=1)
    w = case.weights
    tr = ntc.Trainer(64, 64, 5, 12, 4, 4, 4, case.q0, case.q1, case.val0, case.val1,
                     [w[0], w[2], w[4]], [w[1], w[3], w[5]], 80, ntc.PREC_F32, total_steps=10,
                     interp0=ntc.INTERP_LEARNED)
    target = ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(64, 64, 5, seed=1096)))
    with pytest.raises(ntc.NTCError):
        ntc.ntc_train_step(tr, target, 256, 1)


def test_batch_refuses_a_plan_too_large_for_its_regions():
    a = make_case(seed=93, act=1, out_act=1, interp0=1, **PROFILES[1])
    m, _ = device_material(a, precision=ntc.PREC_F16)
    with pytest.raises(ntc.NTCError) as ei:
        ntc.Batch([m], [128])
    assert ei.value.code == ntc.ERR_UNSUPPORTED
