"""The library's FP8-E4M3 preparation calls (the precision form below the
paper's half precision, Sec. 5.1, 7): ntc_f8_quantize_weights (per-layer
weight scale max|W| / 448 and E4M3 bytes) and ntc_f8_activation_scales
(power-of-two activation scales from an FP32 decode of calibration queries),
against the oracle's E4M3 rounding and the oracle's layer inputs; then the
FP8 material they build decoded against the oracle's FP8 form."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


@pytest.mark.parametrize("rows,cols,cols_out", [(64, 48, 64), (64, 64, 64), (12, 64, 64),
                                                (64, 29, 32), (3, 5, 16)])
def test_quantize_weights_matches_e4m3_rounding(rows, cols, cols_out):
    rng = np.random.default_rng(rows * 1000 + cols)
    w = (rng.standard_normal((rows, cols)) * rng.uniform(0.01, 3.0)).astype(np.float32)
    w[0, 0] = 0.0
    w8, s = ntc.ntc_f8_quantize_weights(torch.from_numpy(w).to(DEV), cols_out)
    s = float(s.item())
    assert s == np.float32(np.abs(w).max()) / np.float32(448.0)
    got = w8.view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
    want = oracle.round_e4m3((w / np.float32(s)).astype(np.float32).astype(np.float64))
    assert np.array_equal(got[:, :cols], want)
    assert not np.any(got[:, cols:])
    assert np.abs(got).max() == 448.0   # the largest weight maps to the top of the range
    z, sz = ntc.ntc_f8_quantize_weights(torch.zeros((4, 8), device=DEV))
    assert float(sz.item()) == 1.0 and not torch.any(z)


def _oracle_layer_maxima(md, q):
    """Largest |input| of each layer over the nearest decodes of q (FP64)."""
    x = md.features_uvl(q)
    w = md.weights
    act = np.vectorize(lambda z: oracle.activation(md.act, z))
    h1 = act(x @ w[0].T + w[1])
    h2 = act(h1 @ w[2].T + w[3])
    return [np.abs(a).max() for a in (x, h1, h2)]


@pytest.mark.parametrize("shape", [
    dict(width=512, height=512, channels=16, c0=12, c1=12, k_in=48),
    dict(width=256, height=256, channels=9, c0=16, c1=8, k_in=64, act=1, out_act=1),
])
def test_activation_scales_match_oracle_maxima(shape):
    case = make_case(seed=121, wgain=4.0, **shape)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = gen.random_queries(20000, md.mips, seed=4121)
    sa = to_np(ntc.ntc_f8_activation_scales(mat, torch.from_numpy(q).to(DEV)))
    for l, a in enumerate(_oracle_layer_maxima(md, q)):
        want = 2.0 ** np.ceil(np.log2(a / 448.0))
        if sa[l] != want:  # only at a power-of-two boundary (FP32 vs FP64 maxima)
            assert abs(np.log2(a / 448.0) - np.round(np.log2(a / 448.0))) < 1e-5, (l, sa[l], want)
        assert a / sa[l] <= 448.0 * (1 + 1e-6)
    # no queries: every scale is 1
    e = torch.empty((0, 3), dtype=torch.float32, device=DEV)
    assert to_np(ntc.ntc_f8_activation_scales(mat, e)).tolist() == [1.0, 1.0, 1.0]


def test_f8_material_decodes_like_the_fp8_oracle():
    """The FP8 material built by the two calls (weights of the FP32 model,
    scales calibrated on other queries) against the oracle's FP8 form with
    the same scales and stored weights; bars as the FP8 decode tests (an
    E4M3 rounding decision can move one input by one step)."""
    case = make_case(512, 512, 16, 12, 12, k_in=48, seed=122)
    mat16, _ = device_material(case, precision=ntc.PREC_F16)
    calib = torch.from_numpy(gen.random_queries(8192, mat16.mips, seed=4122)).to(DEV)
    w32 = [case.weights[l] for l in (0, 2, 4)]
    m8 = ntc.f8_material(mat16, w32, calib)
    sc = to_np(m8.scale)
    stored = []
    for l in range(3):
        wq = m8.weights[l].view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
        stored += [wq[:, :case.weights[2 * l].shape[1]] * sc[l], case.weights[2 * l + 1]]
    md = case.oracle_model(weights=[np.asarray(a, np.float64) for a in stored])
    q = gen.random_queries(4096 + 7, md.mips, seed=4123)
    got = to_np(ntc.ntc_decode(m8, torch.from_numpy(q).to(DEV)))
    assert ntc.ntc_device_status() == ntc.OK
    ref = md.decode_f8(q, list(sc[:3]), list(sc[3:]))
    err = np.abs(got - ref)
    assert np.mean(err <= 2e-3) >= 0.99, np.mean(err <= 2e-3)
    assert err.max() <= 2e-2, err.max()
