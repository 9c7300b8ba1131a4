"""The tensor-core adjoint: ntc_backward on FP16 materials (reverse mode of
the decode, Sec. 4.5) runs the fused training kernel fed an upstream
gradient instead of the loss, and NTCDecodeFunction puts it behind
torch.autograd.  Against the FP64 oracle's reverse mode at 1e-2 relative
error per tensor (the training bar): bilinear and learned G0 (the paper's
decoder: K = 96, hardGELU, identity output), two and three hidden layers,
with and without the quantisation noise, and upstream gradients of very
small and very large magnitude (each CTA rescales them by a power of two
before the FP16 products)."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, check_grads, device_material, to_np

pytestmark = pytest.mark.gpu

CASES = {
    "small": dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32),
    "bench": dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48),
    "odd": dict(width=32, height=64, channels=3, c0=3, c1=5, k_in=32),
    # the paper's decoder at profile 2.25 (Sec. 4.3.1, 4.4, 6)
    "paper": dict(width=256, height=256, channels=9, c0=16, c1=12, k_in=96, act=1, out_act=1,
                  interp0=1),
    "paper3": dict(width=128, height=128, channels=9, c0=12, c1=10, bits0=2, k_in=80, act=1,
                   out_act=1, interp0=1, hidden_layers=3),
    "deep": dict(width=128, height=64, channels=16, c0=12, c1=12, k_in=48, hidden_layers=3),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _texels(md, q):
    m = np.minimum(np.floor(q[:, 2]).astype(np.int64), md.mips - 1)
    wm, hm = np.maximum(1, md.width >> m), np.maximum(1, md.height >> m)
    x = np.minimum(np.floor(q[:, 0] * wm).astype(np.int64), wm - 1)
    y = np.minimum(np.floor(q[:, 1] * hm).astype(np.int64), hm - 1)
    return np.stack([x, y, m], 1).astype(np.int32)


def _zeros_like_params(case):
    g0 = [torch.zeros(v.shape, device=DEV) for v in case.val0]
    g1 = [torch.zeros(v.shape, device=DEV) for v in case.val1]
    w = [torch.zeros(a.shape, device=DEV) for a in case.weights[0::2]]
    b = [torch.zeros(a.shape, device=DEV) for a in case.weights[1::2]]
    return g0, g1, w, b


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("scale,noise", [(1.0, None), (1e-6, (5, 6)), (3e4, None)])
def test_backward_f16_tensor_cores_match_oracle(name, scale, noise):
    case = make_case(seed=101, **CASES[name])
    mat, md = device_material(case, precision=ntc.PREC_F16, packed=False)
    n = 7 * 128 + 51
    q = gen.random_texel_queries(case.width, case.height, md.mips, n, seed=4101)
    rng = np.random.default_rng(102)
    dout = (scale * rng.standard_normal((n, case.channels))).astype(np.float32)
    g0, g1, w, b = _zeros_like_params(case)
    gs = ntc.grads_struct(mat, g0, g1, w, b)
    ntc.ntc_backward(mat, torch.from_numpy(q).to(DEV), torch.from_numpy(dout).to(DEV), gs,
                     flags=ntc.FLAG_NOISE if noise else 0,
                     noise_seed=noise[0] if noise else 0, noise_step=noise[1] if noise else 0)
    assert ntc.ntc_device_status() == ntc.OK
    gref = md.backward_xym(_texels(md, q), dout.astype(np.float64), noise=noise)
    check_grads(g0 + g1 + w + b, gref["grid0"] + gref["grid1"] + gref["w"][0::2] + gref["w"][1::2],
                2 * len(case.val0), True)


@pytest.mark.parametrize("name", ["paper", "paper3"])
def test_autograd_paper_form_f16_matches_oracle(name):
    """decode_autograd on the paper's decoder form with FP16 weights: an L2
    loss through torch autograd, its gradients from the tensor-core adjoint."""
    case = make_case(seed=103, **CASES[name])
    mat, md = device_material(case, precision=ntc.PREC_F16, packed=False)
    n = 5 * 128 + 3
    q = gen.random_texel_queries(case.width, case.height, md.mips, n, seed=4103)
    nl = len(case.weights) // 2
    params = [torch.tensor(a, device=DEV, requires_grad=True)
              for a in case.val0 + case.val1 + case.weights[0::2] + case.weights[1::2]]
    L = len(case.val0)
    y = ntc.decode_autograd(mat, torch.from_numpy(q).to(DEV), params[:L], params[L:2 * L],
                            params[2 * L:2 * L + nl], params[2 * L + nl:], noise=(7, 8))
    tgt = torch.rand(y.shape, device=DEV, generator=torch.Generator(DEV).manual_seed(9))
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    lref, gref = md.loss_grad_xym(_texels(md, q), to_np(tgt), noise=(7, 8))
    assert abs(loss.item() - lref) <= 2e-3 * lref
    check_grads([p.grad for p in params],
                gref["grid0"] + gref["grid1"] + gref["w"][0::2] + gref["w"][1::2], 2 * L, True)
