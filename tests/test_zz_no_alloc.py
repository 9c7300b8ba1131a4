"""The allocation-free optimisation step against the regular one.

ntc_train_step_noalloc serves callers that must not allocate device memory
(frame loops, streams under graph capture, plugins handed their buffers by a
host): its scratch gradient is a static array inside the library.  Both
trainers run through it: the FP32 CUDA-core step and the default FP16
tensor-core step (and its FP8-E4M3 form).  This file is collected last so that a run stopping at its
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import ntc_inputs as gen
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import rel_err

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _trainer(case, precision):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                       [w[1], w[3], w[5]], case.k_in, precision, case.act, case.out_act,
                       total_steps=20)


def _step_both(ref, cand, target, batch, seed, call):
    p_ref0, p_cand0 = ref.params.clone(), cand.params.clone()
    l_ref = ntc.ntc_train_step(ref, target, batch, seed).item()
    l_cand = ntc.ntc_train_step_noalloc(cand, target, batch, seed).item()
    assert ntc.ntc_device_status() == ntc.OK
    assert abs(l_ref - l_cand) <= 1e-6 * max(1.0, l_ref), (call, l_ref, l_cand)
    assert int(ref.step_t.item()) == int(cand.step_t.item())
    d_ref = (ref.params - p_ref0).double().cpu().numpy()
    d_cand = (cand.params - p_cand0).double().cpu().numpy()
    assert np.abs(d_ref).max() > 0
    assert rel_err(d_cand, d_ref) <= GRAD_TOL, call


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16, ntc.PREC_F8])
def test_noalloc_step_matches_regular_step_twice(precision):
    case = make_case(128, 128, 6, 8, 8, k_in=32, seed=61)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 6, seed=1061))
    target = ntc.Target(chain)
    ref, cand = _trainer(case, precision), _trainer(case, precision)
    for call in range(2):
        _step_both(ref, cand, target, 4 * 128 + 9, 321, call)
        assert int(ref.step_t.item()) == call + 1


@pytest.mark.parametrize("precision", [ntc.PREC_F32, ntc.PREC_F16])
def test_noalloc_after_a_larger_material(precision):
    """A step of a larger material through the shared array, then two steps
    of a smaller one: the smaller one's steps equal the regular step's (the
    array is cleared for each call's parameter count)."""
    big = make_case(256, 256, 12, 16, 16, k_in=48, seed=63)
    chain_big = gen.box_mip_chain_u8(gen.synthetic_texture(256, 256, 12, seed=1063))
    tr_big = _trainer(big, precision)
    ntc.ntc_train_step_noalloc(tr_big, ntc.Target(chain_big), 3000, 7)
    assert ntc.ntc_device_status() == ntc.OK
    small = make_case(64, 64, 5, 8, 8, k_in=32, seed=64)
    target = ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(64, 64, 5, seed=1064)))
    ref, cand = _trainer(small, precision), _trainer(small, precision)
    assert cand.params.numel() < tr_big.params.numel()
    for call in range(2):
        _step_both(ref, cand, target, 2 * 128 + 3, 55, call)


def test_noalloc_refuses_gradient_only_steps():
    case = make_case(64, 64, 4, 8, 8, k_in=32, seed=62)
    tr = _trainer(case, ntc.PREC_F16)
    target = ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(64, 64, 4, seed=1062)))
    p0 = tr.params.clone()
    with pytest.raises(ntc.NTCError) as ei:
        ntc.ntc_train_step_noalloc(tr, target, 256, 1, flags=ntc.FLAG_GRAD_ONLY)
    assert ei.value.code == ntc.ERR_ARG
    assert "GRAD_ONLY" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.equal(tr.params, p0) and int(tr.step_t.item()) == 0


def test_noalloc_rejects_too_many_parameters():
    case = make_case(64, 64, 4, 8, 8, k_in=32, seed=62)
    tr = _trainer(case, ntc.PREC_F32)
    target = ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(64, 64, 4, seed=1062)))
    t = tr.struct
    t.n_params = (1 << 21) + 1
    m, tg = tr.material.struct, target.struct
    rc = ntc.lib().ntc_train_step_noalloc(C.byref(m), C.byref(t), C.byref(tg), 64, 1, None,
                                          C.c_void_p(tr.loss.data_ptr()), 0, None)
    assert rc == ntc.ERR_SHAPE
    assert "NTC_NOALLOC_MAX_PARAMS" in ntc.lib().ntc_last_error().decode()
