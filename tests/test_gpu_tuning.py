"""The autotuners and their tuning cache: the decode's launch shape and the
training step's pipelines per CTA, keyed by shape, precision, SM count and
size bucket; the choice is used by later calls with the same key and
survives an export / import round trip."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, check_grads, device_material, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()
    ntc.tuning_clear()
    yield
    ntc.tuning_clear()


def test_decode_autotuner_records_its_choice_per_key():
    case = make_case(512, 512, 16, 12, 12, k_in=48, seed=151)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = gen.random_queries(40000, md.mips, seed=4151)
    uvl = torch.from_numpy(q).to(DEV)
    out = torch.empty((q.shape[0], 16), dtype=torch.float16, device=DEV)
    best, ms = ntc.ntc_autotune_decode(mat, uvl, out)
    assert best in (2, 3, 4, 5) and all(v > 0 for v in ms.values())
    text = ntc.tuning_export()
    lines = [l for l in text.splitlines() if l.startswith("decode:")]
    assert len(lines) == 1 and lines[0].endswith(f" {best}") and ":n=2^15" in lines[0]
    # the next decode with this key uses it, and is still correct
    got = ntc.ntc_decode(mat, uvl, out_dtype=torch.float16).float().cpu().numpy()
    assert ntc.ntc_device_status() == ntc.OK
    assert np.abs(got - md.decode(q)).max() <= 2e-3


@pytest.mark.parametrize("precision", [ntc.PREC_F16, ntc.PREC_F8])
def test_train_autotuner_choice_is_used_and_leaves_state(precision):
    case = make_case(128, 128, 12, 16, 16, k_in=64, seed=152)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(128, 128, 12, seed=1152))
    w = case.weights
    tr = ntc.Trainer(128, 128, 12, 16, 16, 4, 4, case.q0, case.q1, case.val0, case.val1,
                     [w[0], w[2], w[4]], [w[1], w[3], w[5]], 64, precision, total_steps=20,
                     f8_act_scales=[1.0 / 256, 1.0 / 64, 1.0 / 64] if precision == ntc.PREC_F8 else None)
    target = ntc.Target(chain)
    p0 = tr.params.clone()
    sc0 = tr.f8_scale.clone() if tr.f8_scale is not None else None
    best, ms = ntc.ntc_autotune_train(tr, target, 3000, 5)
    assert ntc.ntc_device_status() == ntc.OK
    assert best in (1, 2, 3) and ms[best - 1] > 0 and ms[0] > 0
    assert torch.equal(tr.params, p0) and int(tr.step_t.item()) == 0
    assert float(tr.grad.abs().max()) == 0.0
    if sc0 is not None:
        assert torch.equal(tr.f8_scale, sc0)
    key = [l for l in ntc.tuning_export().splitlines() if l.startswith("train:")
           and f"prec={precision}:" in l]
    assert len(key) == 1 and key[0].endswith(f" {best}")
    # every pipeline count gives the same gradient (up to atomic order); the
    # cached choice runs in the regular step
    grads = []
    for np_choice in sorted({1, best}):
        ntc.tuning_import(key[0].rsplit(" ", 1)[0] + f" {np_choice}")
        tr.grad.zero_()
        tr.step_t.fill_(1)
        ntc.ntc_train_step(tr, target, 3000, 5, flags=ntc.FLAG_GRAD_ONLY)
        assert ntc.ntc_device_status() == ntc.OK
        grads.append(to_np(tr.grad))
    assert np.linalg.norm(grads[0] - grads[-1]) <= 1e-5 * np.linalg.norm(grads[0])


def test_tuning_cache_round_trip():
    ntc.tuning_import("decode:example 4\ntrain:example 2\n")
    text = ntc.tuning_export()
    ntc.tuning_clear()
    assert ntc.tuning_export() == ""
    ntc.tuning_import(text)
    assert ntc.tuning_export() == text
