"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/), closed forms, library routines (scipy, torch)
on special cases, finite differences and brute force.
"""
import math
import os

import numpy as np
import pytest

import ntc_inputs as gen
import oracle
from _cases import make_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- pyramid ---
def test_table1_pyramid_1024():
    rows = _golden_rows("table1_pyramid_1024.txt")
    lv = oracle.pyramid(1024, 1024)
    assert len(lv) == len(rows)
    n_mips = oracle.mips(1024, 1024)
    assert n_mips == 11
    for j, (level, g0, g1, mips) in enumerate(rows):
        assert int(level) == j
        assert lv[j] == ((int(g0), int(g0)), (int(g1), int(g1)))
        for m in map(int, mips.split(",")):
            assert oracle.level_of_mip(m, len(lv)) == j
    # every mip of the chain is served by exactly one level
    assert sorted(sum([list(map(int, r[3].split(","))) for r in rows], [])) == list(range(n_mips))


def test_table5_grid_storage():
    for prof, side, g0, c0, b0, c1, b1, mb, scope in _golden_rows("table5_grid_storage.txt"):
        side, g0 = int(side), int(g0)
        got = oracle.grid_storage_bytes(side, side, int(c0), int(b0), int(c1), int(b1),
                                        all_levels=(scope == "pyramid"), g0_side=g0) / 2 ** 20
        tol = 1e-9 if scope == "level0" else 3e-3
        assert abs(got - float(mb)) <= tol, (prof, side, got, mb)


def test_pyramid_last_level_serves_three_mips_at_4k():
    lv = oracle.pyramid(4096, 4096)
    assert [a[0] for a, _ in lv] == [1024, 256, 64, 16, 4]
    assert [b[0] for _, b in lv] == [512, 128, 32, 8, 2]
    served = [oracle.level_of_mip(m, len(lv)) for m in range(13)]
    assert served == [0, 0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 4]


# ------------------------------------------------------------ random bits ---
def test_splitmix64_published_vectors():
    gamma = 0x9E3779B97F4A7C15
    for n, hx in _golden_rows("splitmix64_vectors.txt"):
        assert oracle.splitmix64(((int(n) - 1) * gamma) % 2 ** 64) == int(hx, 16)


def test_noise_uniform_in_half_bin():
    q = 1.0 / 16
    v = np.array([oracle.noise_value(7, 3, 0, 0, cell, ch, 4, q) for cell in range(2000)
                  for ch in range(4)])
    assert v.min() >= -q / 2 and v.max() < q / 2
    assert abs(v.mean()) < 0.02 * q
    hist, _ = np.histogram(v, bins=8, range=(-q / 2, q / 2))
    exp = v.size / 8
    assert ((hist - exp) ** 2 / exp).sum() < 30  # chi^2, 7 dof
    # a new value for another step, grid or level
    a = oracle.noise_value(7, 3, 0, 0, 5, 1, 4, q)
    assert a != oracle.noise_value(7, 4, 0, 0, 5, 1, 4, q)
    assert a != oracle.noise_value(7, 3, 0, 1, 5, 1, 4, q)
    assert a != oracle.noise_value(7, 3, 1, 0, 5, 1, 4, q)


def test_sampler_lod_law_chi2():
    """LOD = floor(-log4 X) mixed 95/5 with a uniform LOD (Sec. 5.1)."""
    n_mips, batch = 12, 200_000
    xym = oracle.sample_batch(11, 0, batch, 2048, 2048, n_mips)
    counts = np.bincount(xym[:, 2], minlength=n_mips)
    p = oracle.lod_law_probs(n_mips)
    assert abs(p[0] - (0.95 * 0.75 + 0.05 / 12)) < 1e-15
    exp = p * batch
    ok = exp >= 5
    chi2 = (((counts - exp) ** 2 / exp)[ok]).sum()
    assert chi2 < 40, (counts, exp)  # 11 dof: p < 1e-4
    # texels are inside their mip and uniform over it
    w = np.maximum(1, 2048 >> xym[:, 2])
    assert (xym[:, 0] >= 0).all() and (xym[:, 0] < w).all() and (xym[:, 1] < w).all()
    sel = xym[:, 2] == 0
    hx, _ = np.histogram(xym[sel, 0], bins=16, range=(0, 2048))
    e = sel.sum() / 16
    assert ((hx - e) ** 2 / e).sum() < 45


def test_crop_sampler_lod_law_per_batch_chi2():
    """Crops (Sec. 5.1): one LOD per batch, drawn by the same 95/5 law."""
    n_mips, steps = 12, 20_000
    m = np.array([oracle.sample_batch(13, t, 1, 2048, 2048, n_mips, crops=True)[0, 2]
                  for t in range(steps)])
    counts = np.bincount(m, minlength=n_mips)
    exp = oracle.lod_law_probs(n_mips) * steps
    ok = exp >= 5
    chi2 = (((counts - exp) ** 2 / exp)[ok]).sum()
    assert chi2 < 40, (counts, exp)


@pytest.mark.parametrize("w,h,step", [(2048, 1024, 3), (64, 64, 8), (512, 512, 21)])
def test_crop_sampler_structure(w, h, step):
    """Every texel of a batch from one mip; each 256 x 256 crop is a
    contiguous window (row by row) that wraps around the mip's edges."""
    n_mips = int(np.log2(max(w, h))) + 1
    batch = 3 * 65536 + 1000                     # three whole crops and a ragged one
    xym = oracle.sample_batch(5, step, batch, w, h, n_mips, crops=True)
    m = int(xym[0, 2])
    assert (xym[:, 2] == m).all()
    wm, hm = max(1, w >> m), max(1, h >> m)
    i = np.arange(batch)
    cx, cy, k = i % 256, (i // 256) % 256, i // 65536
    x0, y0 = xym[k * 65536, 0], xym[k * 65536, 1]
    assert np.array_equal(xym[:, 0], (x0 + cx) % wm)
    assert np.array_equal(xym[:, 1], (y0 + cy) % hm)
    # a ragged batch is the prefix of a longer one (same counters)
    assert np.array_equal(oracle.sample_batch(5, step, 70000, w, h, n_mips, crops=True), xym[:70000])


def test_crop_sampler_small_mip_repeats_evenly():
    """A mip smaller than the crop tiles it: every texel of an 8 x 4 mip
    appears (256/8) (256/4) times in a whole crop."""
    for step in range(40):
        xym = oracle.sample_batch(17, step, 65536, 32, 16, 6, crops=True)
        m = int(xym[0, 2])
        wm, hm = max(1, 32 >> m), max(1, 16 >> m)
        if wm < 256 and hm < 256:
            cnt = np.bincount(xym[:, 1] * wm + xym[:, 0], minlength=wm * hm)
            assert (cnt == (256 // wm) * (256 // hm)).all(), (m, cnt)


def test_crop_origins_uniform_and_independent():
    """Crop origins uniform over the mip, different crops of a batch drawn
    independently (mip 0 of a 4096^2 texture, 16 crops x 600 steps)."""
    origins = []
    for step in range(600):
        xym = oracle.sample_batch(23, step, 16 * 65536, 4096, 4096, 1, crops=True)
        origins.append(xym[::65536, :2])
    o = np.concatenate(origins)
    hx, _ = np.histogram(o[:, 0], bins=16, range=(0, 4096))
    hy, _ = np.histogram(o[:, 1], bins=16, range=(0, 4096))
    e = len(o) / 16
    assert ((hx - e) ** 2 / e).sum() < 45 and ((hy - e) ** 2 / e).sum() < 45
    r = np.corrcoef(o[:-1, 0], o[1:, 0])[0, 1]
    assert abs(r) < 0.05


def test_e4m3_rounding_by_hand_and_against_torch():
    """E4M3 rounding (OCP FP8: bias 7, 3 mantissa bits, max 448): hand values
    (ties to even, subnormals, saturation), then torch's float8_e4m3fn cast
    on float32 inputs inside the finite range."""
    r = oracle.round_e4m3
    hand = {1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, 2 ** -9: 2 ** -9, 2 ** -10: 0.0,
            3 * 2 ** -11: 2 ** -9, 448.0: 448.0, 500.0: 448.0, 1e9: 448.0, 240.0: 240.0,
            248.0: 256.0, -1.0625: -1.0, 0.0: 0.0, 0.3: 0.3125, 2 ** -6 * 1.0625: 2 ** -6}
    for x, want in hand.items():
        assert float(r(x)) == want, (x, float(r(x)), want)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(200_000) * np.exp2(rng.integers(-12, 9, 200_000))).astype(np.float32)
    x = x[np.abs(x) <= 448.0].astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(r(x), ref)


def test_decode_f8_structure():
    """The FP8 form of the oracle: with the E4M3 rounding replaced by the
    identity the scales cancel and it is the plain decode; with the rounding
    on, each of the three layer inputs (K, 64, 64 values) is rounded once, in
    units of its activation scale."""
    from _cases import make_case
    case = make_case(64, 64, 6, 8, 8, k_in=32, seed=31)
    md = case.oracle_model()
    q = np.random.default_rng(3).random((50, 3)).astype(np.float32)
    q[:, 2] *= md.mips
    s_w, s_a = [0.01, 0.02, 0.03], [1 / 256, 4 / 256, 4 / 256]
    real = oracle.round_e4m3
    calls = []
    try:
        oracle.round_e4m3 = lambda a: (calls.append(np.array(a)), np.asarray(a))[1]
        ident = md.decode_f8(q, s_w, s_a)
    finally:
        oracle.round_e4m3 = real
    assert np.abs(ident - md.decode(q)).max() < 1e-12
    assert [c.shape[1] for c in calls] == [32, 64, 64]
    assert np.abs(calls[0] * s_a[0] - md.features_uvl(q)).max() < 1e-12
    f8 = md.decode_f8(q, s_w, s_a)
    assert 0 < np.abs(f8 - ident).max() < 0.1


def test_c_e4m3_rounding_against_torch():
    """The C oracle's E4M3 rounding (used inside its FP8 forward) against
    torch's float8_e4m3fn cast, bit for bit, and NaN/zero/sign handling."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    x = (rng.standard_normal(50_000) * np.exp2(rng.integers(-14, 10, 50_000))).astype(np.float32)
    x = x[np.abs(x) <= 448.0].astype(np.float64)
    got = np.array([oracle.lib().or_round_e4m3(v) for v in x])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(got, ref)
    assert oracle.lib().or_round_e4m3(1e6) == 448.0 and oracle.lib().or_round_e4m3(-1e6) == -448.0
    assert math.isnan(oracle.lib().or_round_e4m3(float("nan")))
    assert math.copysign(1.0, oracle.lib().or_round_e4m3(-1e-9)) == -1.0


def _f8_model(act, seed=21, out_act=0, interp0=0):
    """A small material, its FP64 model and its FP8 form with power-of-two
    scales: weights max |W| / s_w in (224, 448]; activation scales chosen
    from the FP64 activations so that each layer meets a different part of
    the E4M3 range (layer 0 normal values, layer 1 about 10% saturated,
    layer 2 about half subnormal) -- with power-of-two scales the rounding
    depends on the scale only at the range's ends."""
    case = make_case(32, 32, 4, 4, 4, k_in=48 if interp0 else 32, hidden=16, act=act, seed=seed,
                     wgain=2.0, out_act=out_act, interp0=interp0)
    md = case.oracle_model(quantized=False)
    w = md.weights
    s_w = [float(2.0 ** np.ceil(np.log2(np.abs(w[2 * l]).max() / 448.0))) for l in range(3)]
    x = np.stack([md.features(a, b, m) for a, b, m in _texels(md, 200, seed)])
    f = np.vectorize(lambda z: oracle.activation(act, z))
    h1 = f(x @ w[0].T + w[1])
    h2 = f(h1 @ w[2].T + w[3])
    s_a = [float(2.0 ** np.ceil(np.log2(np.abs(x).max() / 448.0))),
           float(2.0 ** np.floor(np.log2(np.quantile(np.abs(h1), 0.9) / 448.0))),
           float(2.0 ** np.ceil(np.log2(np.quantile(np.abs(h2[h2 != 0]), 0.5) / 2.0 ** -6)))]
    assert len(set(s_a)) == 3
    return md, md.f8_form(s_w, s_a), s_w, s_a


def _texels(md, n, seed):
    rng = np.random.default_rng(seed)
    return np.array([[rng.integers(0, md.width >> m), rng.integers(0, md.height >> m), m]
                     for m in rng.integers(0, md.mips, size=n)], np.int32)


def test_f8_form_forward_matches_python_decode_f8():
    """The C oracle's FP8 forward (rounding inside the MLP) equals the
    separately pinned Python FP8 decode of the same quantised weights, and
    its weights are E4M3 multiples of s_w."""
    md, f8, s_w, s_a = _f8_model(0)
    q = np.random.default_rng(5).random((300, 3)).astype(np.float32)
    q[:, 2] *= md.mips
    a = f8.decode(q)
    b = f8.decode_f8(q, s_w, s_a)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14)
    assert np.abs(a - md.decode(q)).max() > 1e-4          # the rounding is felt
    for l in range(3):
        w = f8.weights[2 * l] / s_w[l]
        assert np.array_equal(oracle.round_e4m3(w), w) and np.abs(w).max() <= 448


@pytest.mark.parametrize("act,out_act,interp0", [(0, 0, 0), (1, 0, 0), (1, 1, 1)])
def test_f8_form_gradients_are_straight_through(act, out_act, interp0):
    """Reverse mode of the FP8 form against torch autograd (float64) of the
    same forward written with the straight-through estimator
    v + (s e4m3(v / s) - v).detach(): loss, every weight and bias gradient,
    and each texel's input-row gradient (ReLU or hardGELU, sigmoid or
    identity output, bilinear or learned G0 rows)."""
    torch = pytest.importorskip("torch")
    md, f8, s_w, s_a = _f8_model(act, out_act=out_act, interp0=interp0)
    xym = _texels(md, 48, 6)
    target = np.random.default_rng(7).random((48, 4))
    noise = (99, 4)
    loss, g = f8.loss_grad_xym(xym, target, noise=noise, rows=True)
    X = torch.tensor(np.stack([f8.features(x, y, m, noise) for x, y, m in xym]),
                     requires_grad=True)
    W = [torch.tensor(w, requires_grad=True) for w in f8.weights]

    def ste(v, s):
        q = torch.from_numpy(s * oracle.round_e4m3(v.detach().numpy() / s))
        return v + (q - v).detach()

    def act_t(z):
        if act == 0:
            return torch.relu(z)
        return torch.where(z < -1.5, torch.zeros_like(z),
                           torch.where(z > 1.5, z, z / 3.0 * (z + 1.5)))

    h = ste(X, s_a[0])
    h = act_t(h @ W[0].T + W[1])
    h = act_t(ste(h, s_a[1]) @ W[2].T + W[3])
    z3 = ste(h, s_a[2]) @ W[4].T + W[5]
    y = z3 if out_act == 1 else torch.sigmoid(z3)
    lt = ((y - torch.from_numpy(target)) ** 2).mean()
    lt.backward()
    assert abs(loss - lt.item()) <= 1e-12 * lt.item()
    for gw, wt in zip(g["w"], W):
        assert np.allclose(gw, wt.grad.numpy(), rtol=1e-9, atol=1e-15)
    assert np.allclose(g["rows"], X.grad.numpy(), rtol=1e-9, atol=1e-15)
    assert np.abs(g["rows"]).max() > 0


def test_f8_form_grid_gradient_is_the_transpose_of_the_features():
    """The grid gradients are the row gradients pulled back through the
    (linear) feature map: <dL/dgrid, d> = sum_i <dL/drow_i, rows_i(grid + d)
    - rows_i(grid)> for a random direction d, noise on."""
    md, f8, s_w, s_a = _f8_model(1, seed=22)
    xym = _texels(md, 40, 8)
    target = np.random.default_rng(9).random((40, 4))
    noise = (7, 3)
    _, g = f8.loss_grad_xym(xym, target, noise=noise, rows=True)
    rng = np.random.default_rng(10)
    grids = f8.grids0 + f8.grids1
    d = [rng.standard_normal(a.shape) for a in grids]
    r0 = np.stack([f8.features(x, y, m, noise) for x, y, m in xym])
    for a, da in zip(grids, d):
        a += da
    r1 = np.stack([f8.features(x, y, m, noise) for x, y, m in xym])
    for a, da in zip(grids, d):
        a -= da
    lhs = sum(np.sum(ga * da) for ga, da in zip(g["grid0"] + g["grid1"], d))
    rhs = np.sum(g["rows"] * (r1 - r0))
    assert abs(lhs - rhs) <= 1e-9 * max(abs(rhs), 1e-12)
    assert abs(rhs) > 0


def test_f8_form_output_layer_matches_central_differences():
    """The output layer's input is rounded before W3 and b3 act, so the loss
    is smooth in them and central differences must equal the reverse mode
    (a weight gradient formed with the unrounded input would not)."""
    md, f8, s_w, s_a = _f8_model(0, seed=23)
    xym = _texels(md, 32, 11)
    target = np.random.default_rng(12).random((32, 4))
    _, g = f8.loss_grad_xym(xym, target)
    h = 1e-6
    for li in (4, 5):
        p, gp = f8.weights[li].reshape(-1), g["w"][li].reshape(-1)
        for k in np.random.default_rng(li).choice(p.size, size=min(p.size, 24), replace=False):
            old = p[k]
            p[k] = old + h
            lp, _ = f8.loss_grad_xym(xym, target)
            p[k] = old - h
            lm, _ = f8.loss_grad_xym(xym, target)
            p[k] = old
            assert abs((lp - lm) / (2 * h) - gp[k]) <= 1e-6 * max(abs(gp[k]), 1e-8), (li, k)


def _train_oracle(f8, steps=300, batch=1024, seed=5):
    """Texture-set PSNR (Eq. 1) before and after `steps` oracle training
    steps (sampler, noise, L2, Adam with cosine rates, clamping) of a tiny
    32^2 x 4 material, in FP64 or in the FP8 training form (weight scales
    2^ceil(log2(max |W| / 448)) each step, activation scales 2^-6)."""
    w_, h_, c_ = 32, 32, 4
    case = make_case(w_, h_, c_, 4, 4, k_in=32, hidden=16, act=0, seed=41)
    chain = gen.box_mip_chain_u8(gen.synthetic_texture(w_, h_, c_, seed=1041))
    n_lv = len(case.val0)
    params = [np.array(a, np.float64) for a in case.val0 + case.val1 + case.weights]
    mom = [np.zeros_like(p) for p in params]
    vel = [np.zeros_like(p) for p in params]
    rng0 = oracle.quant_range(1 << case.bits0, case.q0)
    rng1 = oracle.quant_range(1 << case.bits1, case.q1)
    mips = oracle.mips(w_, h_)

    def model():
        md = oracle.Model(w_, h_, c_, case.c0, case.c1, 1 << case.bits0, 1 << case.bits1,
                          case.q0, case.q1, params[:n_lv], params[n_lv:2 * n_lv],
                          params[2 * n_lv:], case.k_in, 16, 0, 0)
        if not f8:
            return md
        s_w = [float(2.0 ** np.ceil(np.log2(np.abs(params[2 * n_lv + 2 * l]).max() / 448.0)))
               for l in range(3)]
        return md.f8_form(s_w, [2.0 ** -6] * 3)

    def texture_psnr():
        md, ref, dec = model(), [], []
        for m in range(mips):
            ys, xs = np.meshgrid(np.arange(max(1, h_ >> m)), np.arange(max(1, w_ >> m)),
                                 indexing="ij")
            xym = np.stack([xs.ravel(), ys.ravel(), np.full(xs.size, m)], 1).astype(np.int32)
            dec.append(md.decode_xym(xym))
            ref.append(oracle.targets_of_xym(chain, xym))
        return oracle.texture_set_psnr(ref, dec)

    before = texture_psnr()
    for t in range(steps):
        xym = oracle.sample_batch(seed, t, batch, w_, h_, mips)
        _, g = model().loss_grad_xym(xym, oracle.targets_of_xym(chain, xym), noise=(seed, t))
        for i, (p, gr) in enumerate(zip(params, g["grid0"] + g["grid1"] + g["w"])):
            lr = oracle.cosine_lr(1e-2 if i < 2 * n_lv else 5e-3, t, steps)
            clamp = rng0 if i < n_lv else (rng1 if i < 2 * n_lv else None)
            oracle.adam(p, mom[i], vel[i], gr, lr, t + 1, clamp=clamp)
    return before, texture_psnr()


def test_f8_training_form_converges_like_fp64():
    """Training in the FP8 form (straight-through gradients applied to the
    master weights) reaches the FP64 training's quality on a tiny material:
    both gain several dB from the same start, and end within 0.3 dB."""
    b64, a64 = _train_oracle(False)
    b8, a8 = _train_oracle(True)
    assert a64 > b64 + 5.0 and a8 > b8 + 5.0
    assert abs(a8 - a64) < 0.3, (a8, a64)


def test_vq_reconstruct_by_hand():
    """A vector-quantised cell is the sum of the entries its indices select."""
    cb = np.zeros((2, 256, 2))
    cb[0, 3] = [1.0, 2.0]
    cb[1, 7] = [0.25, -0.5]
    cb[1, 0] = [10.0, 10.0]
    idx = np.array([[[3, 7], [3, 0]]], np.uint8)
    got = oracle.vq_reconstruct(idx, cb)
    assert got.shape == (1, 2, 2)
    assert np.array_equal(got[0, 0], [1.25, 1.5]) and np.array_equal(got[0, 1], [11.0, 12.0])


def test_vq_assign_single_book_is_nearest_entry():
    """One codebook: the nearest entry (brute force in float64 on points far
    from any tie)."""
    rng = np.random.default_rng(5)
    cb = rng.integers(-20, 20, size=(1, 256, 4)).astype(np.float32) * 4.0
    cb = np.unique(cb[0], axis=0)[None, :256]
    if cb.shape[1] < 256:
        cb = np.concatenate([cb, np.full((1, 256 - cb.shape[1], 4), 1e4, np.float32)], 1)
    pick = rng.integers(0, 256, 500)
    vals = cb[0, pick] + rng.uniform(-0.5, 0.5, (500, 4)).astype(np.float32)
    want = np.argmin(((vals[:, None, :].astype(np.float64) - cb[0][None]) ** 2).sum(-1), 1)
    assert np.array_equal(oracle.vq_assign(vals, cb)[:, 0], want)


def test_vq_assign_residual_and_ties_by_hand():
    """Two books on a 1-D example: 11.2 -> 10 (book 0) then 1 (book 1);
    equal entries resolve to the lowest index."""
    cb = np.full((2, 256, 1), 1e3, np.float32)
    cb[0, 0], cb[0, 5] = 0.0, 10.0
    cb[1, 0], cb[1, 1], cb[1, 2] = 0.0, 1.0, -1.0
    cb[1, 9] = 1.0                         # a duplicate of entry 1
    idx = oracle.vq_assign(np.array([[11.2], [9.1], [0.2]], np.float32), cb)
    assert idx.tolist() == [[5, 1], [5, 2], [0, 0]]


def test_vq_train_terms_by_hand():
    """VQ-VAE terms on a hand example: one book {0: 0, 1: 1}, latents 0.2 and
    0.9 (N = 2): indices 0, 1; q = 0, 1; codebook gradient 2/N (e - r) =
    -0.2, 0.1; commitment gradient 2 beta/N (z - q) = beta (0.2, -0.1)."""
    cb = np.full((1, 256, 1), 50.0, np.float32)
    cb[0, 0, 0], cb[0, 1, 0] = 0.0, 1.0
    idx, q, dz, dcb = oracle.vq_train_terms([np.array([[[0.2], [0.9]]], np.float32)], cb, 0.25)
    assert idx[0].reshape(-1).tolist() == [0, 1]
    assert np.allclose(q[0].reshape(-1), [0.0, 1.0])
    assert np.allclose(dcb[0, :2, 0], [-0.2, 0.1], atol=1e-7) and not np.any(dcb[0, 2:])
    assert np.allclose(dz[0].reshape(-1), [0.05, -0.025], atol=1e-8)


def test_vq_train_terms_residual_books():
    """Two books: the second book's gradient sees what the first leaves
    (r_1 = z - e_0); gradients sum over the cells that share an entry."""
    cb = np.full((2, 256, 1), 50.0, np.float32)
    cb[0, 3, 0] = 10.0
    cb[1, 4, 0], cb[1, 5, 0] = 1.0, -1.0
    z = np.array([[[11.25], [10.75], [9.25]]], np.float32)       # N = 3
    idx, q, dz, dcb = oracle.vq_train_terms([z], cb, 1.0)
    assert idx[0].reshape(3, 2).tolist() == [[3, 4], [3, 4], [3, 5]]
    assert np.allclose(q[0].reshape(-1), [11.0, 11.0, 9.0])
    # book 0, entry 3: 2/3 * ((10 - 11.25) + (10 - 10.75) + (10 - 9.25))
    assert np.isclose(dcb[0, 3, 0], 2 / 3 * (-1.25 - 0.75 + 0.75))
    # book 1: residuals 1.25, 0.75 -> entry 4; -0.75 -> entry 5
    assert np.isclose(dcb[1, 4, 0], 2 / 3 * ((1 - 1.25) + (1 - 0.75)))
    assert np.isclose(dcb[1, 5, 0], 2 / 3 * (-1 + 0.75))
    assert np.allclose(dz[0].reshape(-1), 2 / 3 * np.array([0.25, -0.25, 0.25]))


# ----------------------------------------------------------- quantisation ---
@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_quantizer_levels_and_roundtrip(bits):
    n = 1 << bits
    q = 1.0 / n
    idx = np.arange(n, dtype=np.int32)
    x = oracle.dequantize(idx, n, q)
    # N levels k*Q, k in [-(N/2-1), N/2]; zero is a level (Sec. 4.2)
    assert np.array_equal(x, (np.arange(n) - (n // 2 - 1)) * q)
    assert 0.0 in x and x[n // 2 - 1] == 0.0
    assert np.array_equal(oracle.quantize(x, n, q), idx)
    lo, hi = oracle.quant_range(n, q)
    assert oracle.quantize(np.array([lo, hi, -10.0, 10.0]), n, q).tolist() == [0, n - 1, 0, n - 1]
    # round half to even: (k + 1/2) Q goes to the even neighbour
    mid = (np.arange(-(n // 2 - 1), n // 2) + 0.5) * q
    k = oracle.quantize(mid, n, q) - (n // 2 - 1)
    assert (k % 2 == 0).all()


def test_pack_layout_by_hand():
    # 3 channels x 4 bits -> 12 bits -> 2 bytes per cell; channel 0 in the
    # low nibble of byte 0
    packed = oracle.pack(np.array([[1, 2, 3], [15, 0, 9]]), 3, 4)
    assert packed.tolist() == [[0x21, 0x03], [0x0F, 0x09]]
    # 12 channels x 4 bits -> 48 bits -> padded to 8 bytes
    assert oracle.cell_bytes(12, 4) == 8 and oracle.cell_bytes(8, 2) == 2
    assert oracle.cell_bytes(8, 4) == 4 and oracle.cell_bytes(20, 4) == 16


@pytest.mark.parametrize("c,bits", [(8, 4), (12, 4), (16, 4), (8, 2), (12, 2), (5, 8), (7, 1)])
def test_pack_roundtrip(c, bits):
    rng = np.random.default_rng(c * 10 + bits)
    idx = rng.integers(0, 1 << bits, size=(257, c)).astype(np.int32)
    assert np.array_equal(oracle.unpack(oracle.pack(idx, c, bits), c, bits), idx)


# -------------------------------------------------- positional encoding ---
def test_positional_encoding_closed_form():
    """Triangle waves equal (2/pi) asin(sin) / (2/pi) asin(cos) of the texel
    phase, periods 8, 4, 2 (Sec. 4.3.2); last value of each axis constant."""
    seen = set()
    for y in range(16):
        for x in range(16):
            pe = oracle.positional_encoding(x, y)
            for a, c in enumerate((x, y)):
                for h in range(3):
                    t = (c + 0.5) / (8 >> h)
                    s_ref = 2 / math.pi * math.asin(math.sin(2 * math.pi * t))
                    c_ref = 2 / math.pi * math.asin(max(-1.0, min(1.0, math.cos(2 * math.pi * t))))
                    assert abs(pe[6 * a + 2 * h] - s_ref) < 1e-9
                    assert abs(pe[6 * a + 2 * h + 1] - c_ref) < 1e-9
                assert pe[6 * a + 5] == 0.0
            assert np.array_equal(pe, oracle.positional_encoding(x % 8, y % 8))
            if x < 8 and y < 8:
                seen.add(tuple(pe))
    assert len(seen) == 64  # every texel of the 8x8 tile has its own code


# --------------------------------------------------------- interpolation ---
def test_features_exact_when_grid_matches_mip():
    """At a mip whose resolution equals the grid's, texel centres land on cell
    centres and the interpolated features are the grid values exactly."""
    case = make_case(256, 256, 8, 8, 8, seed=3)
    md = case.oracle_model()
    # G0 of level 0 is 64x64 = mip 2; G1 32x32 = mip 3
    rng = np.random.default_rng(0)
    for _ in range(50):
        x, y = rng.integers(0, 64, size=2)
        row = md.features(int(x), int(y), 2)
        assert np.array_equal(row[:8], md.grids0[0][y, x])
        x, y = rng.integers(0, 32, size=2)
        row = md.features(int(x), int(y), 3)
        assert np.array_equal(row[8:16], md.grids1[0][y, x])


def test_bilinear_matches_scipy_map_coordinates():
    scipy_nd = pytest.importorskip("scipy.ndimage")
    case = make_case(64, 32, 4, 3, 2, seed=4)   # non-square, odd channel counts
    md = case.oracle_model()
    for m in range(md.mips):
        j = oracle.level_of_mip(m, md.levels)
        wm, hm = max(1, 64 >> m), max(1, 32 >> m)
        for (x, y) in [(0, 0), (wm - 1, hm - 1), (wm // 2, hm // 3), (1 % wm, (hm - 1) // 2)]:
            row = md.features(x, y, m)
            for k, (grid, base) in enumerate(((md.grids0[j], 0), (md.grids1[j], md.c0))):
                gh, gw, c = grid.shape
                px = (x + 0.5) / wm * gw - 0.5
                py = (y + 0.5) / hm * gh - 0.5
                for ch in range(c):
                    ref = scipy_nd.map_coordinates(grid[:, :, ch], [[py], [px]], order=1,
                                                   mode="nearest")[0]
                    assert abs(row[base + ch] - ref) < 1e-12


def test_feature_row_layout():
    case = make_case(128, 128, 4, 8, 8, seed=5)
    md = case.oracle_model()
    row = md.features(13, 6, 1)
    assert row.shape == (32,)
    assert np.array_equal(row[16:28], oracle.positional_encoding(13, 6))
    assert row[28] == 1.0 / (md.mips - 1)
    assert (row[29:] == 0).all()


# ------------------------------------------------------------------- MLP ---
def test_hardgelu_closed_form():
    a = oracle.activation
    assert a(1, -2.0) == 0.0 and a(1, 2.0) == 2.0 and a(1, 0.0) == 0.0
    assert a(1, -0.75) == -0.75 / 3 * 0.75
    assert a(1, 1.5) == 1.5 and a(1, -1.5) == 0.0          # continuous at the joints
    assert abs(a(1, 1.5 - 1e-12) - 1.5) < 1e-11 and abs(a(1, -1.5 + 1e-12)) < 1e-11
    assert a(0, -1.0) == 0.0 and a(0, 0.5) == 0.5


def test_decode_matches_torch_mlp_on_oracle_features():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    for act, out_act in [(0, 0), (1, 0), (0, 1)]:
        case = make_case(128, 64, 5, 4, 6, act=act, out_act=out_act, seed=6)
        md = case.oracle_model()
        xym = np.array([[3, 2, 0], [17, 9, 1], [0, 0, 6], [5, 1, 3]], np.int32)
        out = md.decode_xym(xym)
        w = [torch.tensor(a, dtype=torch.float64) for a in md.weights]
        for i, (x, y, m) in enumerate(xym):
            X = torch.tensor(md.features(int(x), int(y), int(m)))
            h = F.linear(X, w[0], w[1])
            h = F.relu(h) if act == 0 else torch.where(
                h < -1.5, torch.zeros_like(h), torch.where(h > 1.5, h, h / 3 * (h + 1.5)))
            h2 = F.linear(h, w[2], w[3])
            h2 = F.relu(h2) if act == 0 else torch.where(
                h2 < -1.5, torch.zeros_like(h2), torch.where(h2 > 1.5, h2, h2 / 3 * (h2 + 1.5)))
            y_ = F.linear(h2, w[4], w[5])
            if out_act == 0:
                y_ = torch.sigmoid(y_)
            assert np.allclose(out[i], y_.numpy(), rtol=0, atol=1e-13)


def test_constant_grids_give_constant_output():
    case = make_case(64, 64, 6, 4, 4, seed=7)
    g0 = [np.full_like(v, 0.25, dtype=np.float64) for v in case.val0]
    g1 = [np.full_like(v, -0.125, dtype=np.float64) for v in case.val1]
    w = [a.copy() for a in case.weights]
    w[0][:, 8:] = 0.0                           # PE and LOD columns off
    md = oracle.Model(64, 64, 6, 4, 4, 16, 16, 1 / 16, 1 / 16, g0, g1, w, case.k_in)
    xym = np.array([[x, y, m] for m in range(md.mips) for x in range(0, 64 >> m, 3)
                    for y in range(0, 64 >> m, 5)], np.int32)
    out = md.decode_xym(xym)
    X = np.zeros(case.k_in)
    X[:4], X[4:8] = 0.25, -0.125
    h1 = np.maximum(w[0] @ X + w[1], 0)
    h2 = np.maximum(w[2] @ h1 + w[3], 0)
    ref = 1 / (1 + np.exp(-(w[4] @ h2 + w[5])))
    assert np.abs(out - ref[None, :]).max() < 1e-14


def test_query_mapping_nearest():
    case = make_case(64, 64, 3, 4, 4, seed=8)
    md = case.oracle_model()
    xym = np.array([[5, 7, 0], [31, 0, 1], [0, 15, 2], [0, 0, 6]], np.int32)
    ref = md.decode_xym(xym)
    uvl = oracle.uvl_of_xym(xym, 64, 64)
    assert np.array_equal(md.decode(uvl), ref)
    # anywhere inside the texel maps to it
    off = uvl.copy()
    off[:, 0] += np.float32(0.49) / np.maximum(1, 64 >> xym[:, 2])
    assert np.array_equal(md.decode(off), ref)
    # clamps: u = 1 -> last texel, lod beyond the chain -> last mip, NaN -> 0
    q = np.array([[1.0, 1.0, 0.0], [0.5, 0.5, 99.0], [np.nan, 0.0, np.nan]], np.float32)
    got = md.decode(q)
    exp = md.decode_xym(np.array([[63, 63, 0], [0, 0, 6], [0, 0, 0]], np.int32))
    assert np.array_equal(got, exp)


def test_trilinear_reduces_to_nearest_at_texel_centres():
    case = make_case(64, 64, 3, 4, 4, seed=9)
    md = case.oracle_model()
    xym = np.array([[5, 7, 0], [31, 2, 1], [3, 3, 3], [0, 0, 6]], np.int32)
    uvl = oracle.uvl_of_xym(xym, 64, 64)
    assert np.abs(md.decode_trilinear(uvl) - md.decode_xym(xym)).max() < 1e-15
    # half way between two mips: the mean of the two bilinear results
    u = np.array([[0.3, 0.6, 2.5]], np.float32)
    lo = md.decode_trilinear(np.array([[0.3, 0.6, 2.0]], np.float32))
    hi = md.decode_trilinear(np.array([[0.3, 0.6, 3.0]], np.float32))
    assert np.abs(md.decode_trilinear(u) - 0.5 * (lo + hi)).max() < 1e-12


def test_learned_interpolation_row_layout():
    """Learned interpolation of G0 (Sec. 4.3.1): the input row holds the four
    neighbouring G0 feature vectors (taps (x0,y0), (x1,y0), (x0,y1), (x1,y1)
    of the bilinear footprint) unweighted, then bilinear G1, PE and LOD; the
    bilinear G0 value is their combination with the bilinear weights."""
    case = make_case(64, 64, 3, 4, 6, k_in=48, seed=14, interp0=1)
    learned = case.oracle_model()
    case.interp0 = 0
    bil = case.oracle_model()
    for x, y, m in [(5, 7, 0), (30, 2, 1), (3, 3, 2), (0, 0, 3)]:
        r4 = learned.features(x, y, m)
        r1 = bil.features(x, y, m)
        taps = r4[:16].reshape(4, 4)
        wm = 64 >> m
        g0 = case.idx0[0].shape[1]
        p = (x + 0.5) / wm * g0 - 0.5
        py = (y + 0.5) / wm * g0 - 0.5
        fx, fy = p - np.floor(p), py - np.floor(py)
        w = np.array([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
        assert np.allclose(w @ taps, r1[:4], atol=1e-12)
        assert np.array_equal(r4[16:16 + 6 + 13], r1[4:4 + 6 + 13])


def test_learned_interpolation_gradients_match_central_differences():
    case = make_case(16, 16, 3, 2, 2, k_in=32, hidden=8, act=1, seed=15, wgain=2.0, interp0=1)
    md = case.oracle_model(quantized=False)
    xym = np.array([[3, 5, 0], [1, 2, 1], [0, 1, 2]], np.int32)
    dout = np.random.default_rng(16).standard_normal((3, 3))
    g = md.backward_xym(xym, dout, noise=(3, 1))
    params = md.grids0 + md.grids1 + md.weights
    grads = g["grid0"] + g["grid1"] + g["w"]
    rng = np.random.default_rng(17)
    for p, gp in zip(params, grads):
        for _ in range(3):
            i = tuple(rng.integers(0, s) for s in p.shape)
            old = p[i]
            p[i] = old + 1e-6
            hi = (md.decode_xym(xym, noise=(3, 1)) * dout).sum()
            p[i] = old - 1e-6
            lo = (md.decode_xym(xym, noise=(3, 1)) * dout).sum()
            p[i] = old
            assert abs((hi - lo) / 2e-6 - gp[i]) <= 1e-6 * max(1.0, abs(gp[i])), (p.shape, i)


def test_stochastic_filter_is_nearest_at_texel_centres():
    """Stochastic filtering (Sec. 5.3) at texel centres with integer LODs: the
    jitter xi in [0, 1) never leaves the texel or the mip, for any frame."""
    case = make_case(64, 32, 3, 4, 4, seed=11)
    md = case.oracle_model()
    xym = np.array([[5, 7, 0], [31, 2, 1], [3, 3, 3], [0, 0, 5], [63, 31, 0]], np.int32)
    uvl = oracle.uvl_of_xym(xym, 64, 32)
    ref = md.decode_xym(xym)
    for step in (0, 1, 77):
        assert np.abs(md.decode_stochastic(uvl, 5, step) - ref).max() == 0.0


def test_stochastic_filter_converges_to_trilinear():
    """Averaged over frames the stochastic decode is the trilinear filter (the
    jitter picks each of the 8 texels with its trilinear weight): the mean of
    400 frames lies within 5 standard errors of the trilinear decode, while
    single frames do not equal it."""
    case = make_case(64, 64, 3, 4, 4, seed=12)
    md = case.oracle_model()
    rng = np.random.default_rng(13)
    q = np.empty((40, 3), np.float32)
    q[:, :2] = rng.random((40, 2))
    q[:, 2] = rng.uniform(0.0, md.mips - 1.0, 40)
    frames = np.stack([md.decode_stochastic(q, 21, s) for s in range(400)])
    mean, se = frames.mean(0), frames.std(0) / np.sqrt(len(frames))
    tri = md.decode_trilinear(q)
    assert np.all(np.abs(mean - tri) <= 5 * se + 1e-12)
    assert np.abs(frames[0] - tri).max() > 1e-3
    # frames are reproducible and differ from one another
    assert np.array_equal(md.decode_stochastic(q, 21, 3), frames[3])
    assert not np.array_equal(frames[3], frames[4])


# ------------------------------------------------------------- gradients ---
def _flat_params(md):
    return md.grids0 + md.grids1 + md.weights


@pytest.mark.parametrize("act,hidden_layers", [(1, 2), (0, 2), (1, 3), (0, 3)])
def test_gradients_match_central_differences(act, hidden_layers):
    """Reverse-mode gradients vs central differences (h = 1e-6) on a tiny
    material with the simulated-quantisation noise switched on, two or three
    hidden layers."""
    case = make_case(16, 16, 3, 2, 2, k_in=32, hidden=8, act=act, seed=10, wgain=2.0,
                     hidden_layers=hidden_layers)
    md = case.oracle_model(quantized=False)
    rng = np.random.default_rng(1)
    xym = np.array([[rng.integers(0, 16 >> m), rng.integers(0, 16 >> m), m]
                    for m in rng.integers(0, md.mips, size=24)], np.int32)
    target = rng.random((24, 3))
    noise = (99, 4)
    loss, g = md.loss_grad_xym(xym, target, noise=noise)
    grads = g["grid0"] + g["grid1"] + g["w"]
    params = _flat_params(md)
    h = 1e-6
    for p, gp in zip(params, grads):
        flat, gflat = p.reshape(-1), gp.reshape(-1)
        num = np.zeros(min(flat.size, 40))
        picks = rng.choice(flat.size, size=num.size, replace=False)
        for i, k in enumerate(picks):
            old = flat[k]
            flat[k] = old + h
            lp, _ = md.loss_grad_xym(xym, target, noise=noise)
            flat[k] = old - h
            lm, _ = md.loss_grad_xym(xym, target, noise=noise)
            flat[k] = old
            num[i] = (lp - lm) / (2 * h)
        ana = gflat[picks]
        err = np.linalg.norm(ana - num) / max(np.linalg.norm(num), 1e-30)
        assert err < 1e-6, (p.shape, err)
    assert loss > 0


def test_third_hidden_layer_reduces_to_two():
    """Three hidden layers whose third is the identity (ReLU, W = I, b = 0;
    h2 >= 0 passes unchanged) decode exactly like the two-layer model, and
    their gradients agree: the third layer's input gradient is the two-layer
    model's, and its weight gradient is the outer product dz h2^T."""
    case = make_case(32, 32, 4, 4, 4, k_in=32, hidden=16, act=0, seed=13)
    md2 = case.oracle_model(quantized=False)
    w = [np.asarray(a, np.float64) for a in case.weights]
    md3 = case.oracle_model(weights=w[:4] + [np.eye(16), np.zeros(16)] + w[4:], quantized=False)
    assert md3.hidden_layers == 3 and md2.hidden_layers == 2
    rng = np.random.default_rng(4)
    xym = np.array([[rng.integers(0, 32 >> m), rng.integers(0, 32 >> m), m]
                    for m in rng.integers(0, md2.mips, size=40)], np.int32)
    assert np.array_equal(md3.decode_xym(xym), md2.decode_xym(xym))
    dout = rng.standard_normal((40, 4))
    g2, g3 = md2.backward_xym(xym, dout), md3.backward_xym(xym, dout)
    for a, b in zip(g2["grid0"] + g2["grid1"] + g2["w"][:4] + g2["w"][4:],
                    g3["grid0"] + g3["grid1"] + g3["w"][:4] + g3["w"][6:]):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)
    assert np.any(g3["w"][4] != 0) and np.any(g3["w"][5] != 0)


def test_backward_is_vector_jacobian_product():
    """Backward of dout equals the directional derivative <dout, dy/dtheta>."""
    case = make_case(32, 32, 4, 4, 4, hidden=16, act=1, seed=12)
    md = case.oracle_model(quantized=False)
    rng = np.random.default_rng(2)
    xym = np.array([[rng.integers(0, 32 >> m), rng.integers(0, 32 >> m), m]
                    for m in rng.integers(0, md.mips, size=10)], np.int32)
    dout = rng.standard_normal((10, 4))
    g = md.backward_xym(xym, dout)
    params = _flat_params(md)
    grads = g["grid0"] + g["grid1"] + g["w"]
    direction = [rng.standard_normal(p.shape) for p in params]
    h = 1e-6
    for p, d in zip(params, direction):
        p += h * d
    yp = md.decode_xym(xym)
    for p, d in zip(params, direction):
        p -= 2 * h * d
    ym = md.decode_xym(xym)
    for p, d in zip(params, direction):
        p += h * d
    num = np.sum(dout * (yp - ym)) / (2 * h)
    ana = sum(np.sum(gr * d) for gr, d in zip(grads, direction))
    assert abs(num - ana) <= 1e-6 * abs(num)


# ------------------------------------------------------------- optimiser ---
def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    p = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    for t in range(6):
        g = rng.standard_normal(50)
        oracle.adam(p, m, v, g, 0.01, t)
        tp.grad = torch.tensor(g)
        opt.step()
        assert np.abs(p - tp.detach().numpy()).max() < 1e-14


def test_adam_first_step_is_sign_and_clamps():
    p = np.array([0.0, 0.0, 0.45, -0.45])
    g = np.array([3.0, -0.2, -1.0, 1.0])
    oracle.adam(p, np.zeros(4), np.zeros(4), g, 0.1, 0, clamp=(-7.5 / 16, 0.5))
    assert np.allclose(p, [-0.1, 0.1, 0.5, -7.5 / 16], atol=1e-7)


def test_cosine_lr():
    assert oracle.cosine_lr(0.01, 0, 100) == 0.01
    assert abs(oracle.cosine_lr(0.01, 50, 100) - 0.005) < 1e-18
    assert abs(oracle.cosine_lr(0.01, 100, 100)) < 1e-18


# ---------------------------------------------------------------- metric ---
def test_texture_set_psnr_eq1():
    ref = [np.zeros((4, 4, 1)), np.zeros((2, 2, 1))]
    test = [np.full((4, 4, 1), 0.1), np.full((2, 2, 1), 0.2)]
    # (16 * 0.01 + 4 * 0.04) / 20 = 0.016
    assert abs(oracle.texture_set_psnr(ref, test) - (-10 * math.log10(0.016))) < 1e-12


def test_oracle_struct_layouts_match_its_header():
    """The oracle's ctypes structs against oracle/ntc_oracle.h compiled by the
    host C compiler: sizeof and every field offset."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pairs = [(oracle._Model, "or_model"), (oracle._Noise, "or_noise"), (oracle._Grads, "or_grads")]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ntc_oracle.h"',
             "int main(void) {"]
    for st, nm in pairs:
        lines.append(f'  printf("{nm} sizeof %zu\\n", sizeof({nm}));')
        for f in st._fields_:
            lines.append(f'  printf("{nm} {f[0]} %zu\\n", offsetof({nm}, {f[0]}));')
    lines += ["  return 0;", "}"]
    out_dir = os.path.join(root, "_build")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "oracle_layout.c"), os.path.join(out_dir, "oracle_layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "oracle"), src, "-o", exe], check=True)
    got = {}
    for line in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for st, nm in pairs:
        assert got[(nm, "sizeof")] == C.sizeof(st), nm
        for f in st._fields_:
            assert got[(nm, f[0])] == getattr(st, f[0]).offset, (nm, f[0])


def test_oracle_signatures_match_its_header():
    """The oracle binding's ctypes argtypes/restypes against the prototypes
    of oracle/ntc_oracle.h."""
    import ctypes as C
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "ntc_oracle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    kinds = {"int": C.c_int, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
             "void": None}
    protos = re.findall(r"([A-Za-z_][\w ]*?)\s+\b(or_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src,
                        flags=re.S)
    assert {p[1] for p in protos} == set(oracle.SIGNATURES)
    for ret, name, params in protos:
        res, args = oracle.SIGNATURES[name]
        assert res is kinds[ret.split()[-1]], name
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        assert len(ps) == len(args), name
        for p, a in zip(ps, args):
            if "*" in p:
                assert a is C.c_void_p, (name, p)
            else:
                t = re.sub(r"\s*\b\w+$", "", p).replace("const ", "").strip()
                assert a is kinds[t], (name, p, a)
