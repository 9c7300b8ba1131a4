"""GPU parity of the FP32 CUDA-core path, the sampler, the quantiser and the
training step against the FP64 oracle (through the C ABI).

Tolerances: decoded values (in [0, 1] after the sigmoid) max-abs 2e-3;
gradients 1e-2 relative (L2 norm of the error over the L2 norm of the
oracle's gradient, per tensor); integer results (quantisation indices, packed
bytes, sampled texels) bit-exact.
"""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case, case_small_fp32, case_train_2k
from _gpu import DEV, device_material, rel_err, to_np

pytestmark = pytest.mark.gpu

OUT_TOL = 2e-3
GRAD_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


# ------------------------------------------------------------------ decode ---
@pytest.mark.parametrize("shape", [
    dict(width=256, height=256, channels=8, c0=8, c1=8, q0=0.125, q1=0.125, k_in=32),
    dict(width=64, height=32, channels=5, c0=4, c1=6, k_in=32, act=1),
    dict(width=128, height=128, channels=16, c0=12, c1=12, k_in=48),
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48, out_act=1),
    dict(width=32, height=32, channels=3, c0=3, c1=2, bits0=2, bits1=8, k_in=32),
    dict(width=64, height=64, channels=4, c0=8, c1=8, k_in=128),
])
def test_decode_fp32_matches_oracle(shape):
    case = make_case(seed=21, **shape)
    mat, md = device_material(case)
    n = 5 * 128 + 37   # several tiles and a ragged tail
    q = gen.random_queries(n, md.mips, seed=4021)
    q[:3] = [[0.0, 0.0, 0.0], [0.999999, 0.999999, md.mips - 1], [0.5, 0.25, 2.0]]
    got = to_np(ntc.ntc_decode(mat, _uvl(q)))
    ref = md.decode(q)
    err = np.abs(got - ref).max()
    assert err <= OUT_TOL, err
    assert err < 1e-5  # FP32 arithmetic lands far inside the bar


def test_decode_edge_cases():
    case = make_case(64, 64, 4, 8, 8, k_in=32, seed=22)
    mat, md = device_material(case)
    # n == 0 is a no-op; NaN / out-of-range coordinates clamp like the oracle
    assert ntc.ntc_decode(mat, _uvl(np.zeros((0, 3)))).shape == (0, 4)
    q = np.array([[np.nan, 0.5, 1.0], [-3.0, 7.0, -1.0], [1.0, 1.0, 99.0], [0.5, 0.5, np.nan],
                  [0.25, 0.75, 6.5]], np.float32)
    got = to_np(ntc.ntc_decode(mat, _uvl(q)))
    assert np.abs(got - md.decode(q)).max() < 1e-5
    # one query
    got1 = to_np(ntc.ntc_decode(mat, _uvl(q[2:3])))
    assert np.abs(got1 - md.decode(q[2:3])).max() < 1e-5
    # a 1x1 texture: one mip, LOD input 0
    c1 = make_case(1, 1, 2, 4, 4, k_in=32, seed=23)
    m1, o1 = device_material(c1)
    q1 = np.array([[0.3, 0.7, 0.0], [0.9, 0.1, 5.0]], np.float32)
    assert np.abs(to_np(ntc.ntc_decode(m1, _uvl(q1))) - o1.decode(q1)).max() < 1e-5


def test_decode_fp16_output():
    case = case_small_fp32(seed=24)
    mat, md = device_material(case)
    q = gen.random_queries(1000, md.mips, seed=4024)
    got = to_np(ntc.ntc_decode(mat, _uvl(q), out_dtype=torch.float16))
    assert np.abs(got - md.decode(q)).max() <= OUT_TOL


def test_decode_f32_grids_and_noise():
    case = make_case(128, 128, 6, 8, 8, k_in=32, seed=25)
    mat, md = device_material(case, packed=False)
    q = gen.random_queries(700, md.mips, seed=4025)
    got = to_np(ntc.ntc_decode(mat, _uvl(q)))
    assert np.abs(got - md.decode(q)).max() < 1e-5
    got_n = to_np(ntc.ntc_decode(mat, _uvl(q), flags=ntc.FLAG_NOISE, noise_seed=77, noise_step=5))
    ref_n = md.decode(q, noise=(77, 5))
    assert np.abs(got_n - ref_n).max() < 1e-5
    assert np.abs(ref_n - md.decode(q)).max() > 1e-4  # the noise is really there


def test_trilinear_matches_oracle():
    case = make_case(128, 64, 5, 8, 8, k_in=32, seed=26)
    mat, md = device_material(case)
    rng = np.random.default_rng(5)
    q = np.empty((300, 3), np.float32)
    q[:, :2] = rng.random((300, 2))
    q[:, 2] = rng.uniform(-0.5, md.mips + 0.5, 300)
    got = to_np(ntc.ntc_decode(mat, _uvl(q), filter=ntc.FILTER_TRILINEAR))
    assert np.abs(got - md.decode_trilinear(q)).max() < 1e-5


def test_sample_features_match_oracle_rows():
    case = make_case(256, 128, 7, 12, 12, k_in=48, seed=27)
    mat, md = device_material(case)
    q = gen.random_queries(400, md.mips, seed=4027)
    rows = to_np(ntc.ntc_sample_features(mat, _uvl(q)))
    for i in range(0, 400, 7):
        x, y, m = _texel(md, q[i])
        ref = md.features(x, y, m)
        assert np.abs(rows[i] - ref).max() < 1e-6
        # positional encoding, LOD and padding are exact
        assert np.array_equal(rows[i][24:], ref[24:].astype(np.float32))


def _texel(md, qrow):
    u, v, l = (float(a) for a in qrow)
    m = 0 if not l >= 0 else min(int(np.floor(l)), md.mips - 1)
    wm, hm = max(1, md.width >> m), max(1, md.height >> m)
    x = min(max(int(np.floor(u * wm)), 0), wm - 1)
    y = min(max(int(np.floor(v * hm)), 0), hm - 1)
    return x, y, m


# ------------------------------------------------------- integer paths -----
@pytest.mark.parametrize("c,bits", [(8, 4), (12, 4), (16, 4), (8, 2), (12, 2), (3, 8), (7, 1)])
def test_quantize_pack_bit_exact(c, bits):
    n = 1 << bits
    q = 1.0 / n
    rng = np.random.default_rng(c + bits)
    lo, hi = oracle.quant_range(n, q)
    x = rng.uniform(lo - 0.1, hi + 0.1, size=(3001, c)).astype(np.float32)
    x[:5, 0] = (np.arange(5) - 2 + 0.5) * q   # exact ties -> even
    idx_ref = oracle.quantize(x.astype(np.float64), n, q)
    packed_ref = oracle.pack(idx_ref, c, bits)
    xt = _uvl(x)
    snapped = torch.empty_like(xt)
    packed = ntc.ntc_quantize_pack(xt, c, bits, q, snapped=snapped)
    assert np.array_equal(packed.cpu().numpy(), packed_ref)
    assert np.array_equal(snapped.cpu().numpy().astype(np.float64), oracle.dequantize(idx_ref, n, q))
    idx, val = ntc.ntc_unpack(packed, c, bits, q)
    assert np.array_equal(idx.cpu().numpy(), idx_ref)
    assert np.array_equal(val.cpu().numpy().astype(np.float64), oracle.dequantize(idx_ref, n, q))


@pytest.mark.parametrize("w,h,step", [(2048, 2048, 0), (256, 64, 17), (4096, 4096, 123456)])
def test_sampler_bit_exact(w, h, step):
    mips = oracle.mips(w, h)
    got = ntc.ntc_sample_batch(99, step, 5000, w, h, mips).cpu().numpy()
    assert np.array_equal(got, oracle.sample_batch(99, step, 5000, w, h, mips))


@pytest.mark.parametrize("w,h,step,batch", [(2048, 2048, 0, 5000), (256, 64, 17, 2 * 65536 + 777),
                                            (4096, 4096, 123456, 4 * 65536), (16, 8, 5, 65536)])
def test_crop_sampler_bit_exact(w, h, step, batch):
    mips = oracle.mips(w, h)
    for s in (step, step + 1, step + 2):
        got = ntc.ntc_sample_batch(99, s, batch, w, h, mips, crops=True).cpu().numpy()
        assert np.array_equal(got, oracle.sample_batch(99, s, batch, w, h, mips, crops=True))


# -------------------------------------------------------------- backward ---
def _grad_views(case, dev=DEV):
    g0 = [torch.zeros(v.shape, dtype=torch.float32, device=dev) for v in case.val0]
    g1 = [torch.zeros(v.shape, dtype=torch.float32, device=dev) for v in case.val1]
    w = [torch.zeros(case.weights[i].shape, dtype=torch.float32, device=dev) for i in (0, 2, 4)]
    b = [torch.zeros(case.weights[i].shape, dtype=torch.float32, device=dev) for i in (1, 3, 5)]
    return g0, g1, w, b


def _check_grads(case, g0, g1, w, b, gref):
    for j in range(len(case.val0)):
        for got, ref in ((g0[j], gref["grid0"][j]), (g1[j], gref["grid1"][j])):
            r = ref.reshape(got.shape)
            if np.linalg.norm(r) > 0:
                assert rel_err(to_np(got), r) <= GRAD_TOL
    for l in range(3):
        assert rel_err(to_np(w[l]), gref["w"][2 * l]) <= GRAD_TOL
        assert rel_err(to_np(b[l]), gref["w"][2 * l + 1]) <= GRAD_TOL


@pytest.mark.parametrize("shape,noise", [
    (dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32), None),
    (dict(width=128, height=64, channels=12, c0=16, c1=16, k_in=48, act=1), (5, 9)),
    (dict(width=32, height=32, channels=3, c0=2, c1=3, k_in=32, out_act=1), (1, 0)),
    (dict(width=64, height=64, channels=8, c0=12, c1=12, k_in=64), None),
])
def test_backward_fp32_matches_oracle(shape, noise):
    case = make_case(seed=31, **shape)
    mat, md = device_material(case, packed=False)
    n = 3 * 128 + 51
    q = gen.random_texel_queries(case.width, case.height, md.mips, n, seed=4031)
    rng = np.random.default_rng(31)
    dout = rng.standard_normal((n, case.channels)).astype(np.float32)
    g0, g1, w, b = _grad_views(case)
    gs = ntc.grads_struct(mat, g0, g1, w, b)
    flags = ntc.FLAG_NOISE if noise else 0
    ntc.ntc_backward(mat, _uvl(q), _uvl(dout), gs, flags=flags,
                     noise_seed=noise[0] if noise else 0, noise_step=noise[1] if noise else 0)
    xym = np.array([_texel(md, r) for r in q], np.int32)
    gref = md.backward_xym(xym, dout.astype(np.float64), noise=noise)
    _check_grads(case, g0, g1, w, b, gref)


def test_autograd_function_matches_oracle():
    case = make_case(64, 64, 4, 8, 8, k_in=32, act=1, seed=33)
    mat, md = device_material(case, packed=False)
    q = gen.random_texel_queries(64, 64, md.mips, 300, seed=4033)
    params = [torch.tensor(a, device=DEV, requires_grad=True)
              for a in case.val0 + case.val1 + [case.weights[i] for i in (0, 2, 4, 1, 3, 5)]]
    L = len(case.val0)
    y = ntc.decode_autograd(mat, _uvl(q), params[:L], params[L:2 * L], params[2 * L:2 * L + 3],
                            params[2 * L + 3:], noise=(3, 4))
    tgt = torch.rand_like(y)
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    xym = np.array([_texel(md, r) for r in q], np.int32)
    lref, gref = md.loss_grad_xym(xym, to_np(tgt), noise=(3, 4))
    assert abs(loss.item() - lref) < 1e-5
    order = gref["grid0"] + gref["grid1"] + [gref["w"][i] for i in (0, 2, 4, 1, 3, 5)]
    for p, r in zip(params, order):
        assert rel_err(to_np(p.grad), r) <= GRAD_TOL


# ------------------------------------------------------------ train step ---
def _trainer_for(case, precision=ntc.PREC_F32, total=100):
    w = case.weights
    return ntc.Trainer(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, case.val0, case.val1, [w[0], w[2], w[4]],
                       [w[1], w[3], w[5]], case.k_in, precision, case.act, case.out_act,
                       total_steps=total)


@pytest.mark.parametrize("shape", [
    dict(width=64, height=64, channels=6, c0=8, c1=8, k_in=32),
    dict(width=128, height=128, channels=12, c0=16, c1=16, k_in=48),
])
def test_train_step_fp32_matches_oracle(shape):
    """Sampler, noise, loss, gradients and one Adam step (+ clamp) against
    the oracle composing the same steps in FP64."""
    case = make_case(seed=41, **shape)
    tex = gen.synthetic_texture(case.width, case.height, case.channels, seed=1041)
    chain = gen.box_mip_chain_u8(tex)
    tr = _trainer_for(case, total=50)
    target = ntc.Target(chain)
    batch, seed = 3 * 128 + 17, 1234
    tr.step_t.fill_(7)
    p0 = tr.params.clone()
    loss = ntc.ntc_train_step(tr, target, batch, seed).item()
    assert int(tr.step_t.item()) == 8
    # oracle: same texels, same noise, FP64 gradients
    md = case.oracle_model(quantized=False)
    xym = oracle.sample_batch(seed, 7, batch, case.width, case.height, md.mips)
    t = oracle.targets_of_xym(chain, xym)
    lref, gref = md.loss_grad_xym(xym, t, noise=(seed, 7))
    assert abs(loss - lref) <= 1e-5 * max(1.0, lref)
    # Adam from zero moments at t = 7: p -= lr_t * g/|g| (bias-corrected) unless g tiny
    gflat = gref["grid0"] + gref["grid1"] + gref["w"]
    L = len(case.val0)
    p_new = tr.params.cpu().numpy().astype(np.float64)
    p_old = p0.cpu().numpy().astype(np.float64)
    for k, (v, g) in enumerate(zip(tr.grad_views, gflat)):
        size = v.numel()
        off = (v.data_ptr() - tr.grad.data_ptr()) // 4
        p = p_old[off:off + size].copy()
        m, vv = np.zeros(size), np.zeros(size)
        grid = k < 2 * L
        lr = oracle.cosine_lr(0.01 if grid else 0.005, 7, 50)
        if grid:
            nq = case.n0 if k < L else case.n1
            qq = case.q0 if k < L else case.q1
            oracle.adam(p, m, vv, g.reshape(-1), lr, 7, clamp=oracle.quant_range(nq, qq))
        else:
            oracle.adam(p, m, vv, g.reshape(-1), lr, 7)
        got = p_new[off:off + size]
        # Adam's first step has magnitude lr wherever |g| >> eps: compare the
        # update itself, which is robust to the gradient's summation order
        upd_ref, upd_got = p - p_old[off:off + size], got - p_old[off:off + size]
        big = np.abs(g.reshape(-1)) > 1e-5
        assert rel_err(upd_got[big], upd_ref[big]) <= GRAD_TOL
    assert float(tr.grad.abs().max()) == 0.0  # scratch gradient left zeroed


def test_train_loop_reduces_loss():
    case = make_case(64, 64, 4, 8, 8, k_in=32, seed=43)
    tex = gen.synthetic_texture(64, 64, 4, seed=1043)
    tr = _trainer_for(case, total=200)
    target = ntc.Target(gen.box_mip_chain_u8(tex))
    losses = [ntc.ntc_train_step(tr, target, 2048, 7).item() for _ in range(200)]
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    lo, hi = oracle.quant_range(16, 1 / 16)
    g = tr.material.grids0[0]
    assert float(g.min()) >= lo - 1e-7 and float(g.max()) <= hi + 1e-7


def test_stochastic_filter_fp32_matches_oracle():
    """FP32 form of the stochastic filter: same texel choice as the oracle,
    outputs within FP32 rounding."""
    case = make_case(128, 64, 5, 6, 10, bits0=2, bits1=8, k_in=32, seed=62)
    mat, md = device_material(case)
    rng = np.random.default_rng(62)
    q = np.empty((2000, 3), np.float32)
    q[:, :2] = rng.uniform(-2.0, 3.0, (2000, 2))
    q[:, 2] = rng.uniform(-1.0, md.mips + 1.0, 2000)
    for seed, step in ((3, 0), (3, 5)):
        got = to_np(ntc.ntc_decode(mat, torch.from_numpy(q).cuda(), filter=ntc.FILTER_STOCHASTIC,
                                   noise_seed=seed, noise_step=step))
        assert np.abs(got - md.decode_stochastic(q, seed, step)).max() < 1e-5
