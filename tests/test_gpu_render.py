"""Render-like precision sweep (the camera workload at reduced size).

A model trained by the library (fused tensor-core steps) is exported with
4-bit packed grids (final quantisation, Sec. 4.2) and decoded with trilinear
filtering (Sec. 5.3) at the queries of a camera over a textured plane, in
FP32 (CUDA cores), FP16 and FP8-E4M3 (tensor cores).  Each is compared with
the FP64 oracle of the same exported model, whose decoder weights are the
FP32 masters: the PSNR then measures the whole precision loss of the form.
The FP16 form is also held to the element-wise bar against the oracle fed
its stored FP16 weights.
"""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _gpu import DEV, to_np

pytestmark = pytest.mark.gpu
SIDE, C, C0, K = 256, 8, 12, 48
Q = 1.0 / 16


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()
    rng = np.random.default_rng(321)
    lo, hi = oracle.quant_range(16, Q)
    g0, g1 = [], []
    for (w0, h0), (w1, h1) in oracle.pyramid(SIDE, SIDE):
        g0.append(gen.uniform_grid_values((h0, w0, C0), lo, hi, rng))
        g1.append(gen.uniform_grid_values((h1, w1, C0), lo, hi, rng))
    w = gen.random_mlp(K, 64, C, seed=322, n_used=2 * C0 + 13)
    steps = 400
    tr = ntc.Trainer(SIDE, SIDE, C, C0, C0, 4, 4, Q, Q, g0, g1, [w[0], w[2], w[4]],
                     [w[1], w[3], w[5]], K, ntc.PREC_F16, total_steps=steps)
    target = ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(SIDE, SIDE, C, seed=323)))
    for _ in range(steps):
        ntc.ntc_train_step(tr, target, 4096, 324)
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    return tr


def _oracle_model(mat, weights):
    """The oracle's model of an exported material: indices unpacked and
    dequantised by the oracle, the given float64 decoder weights."""
    def grids(gs, c):
        out = []
        for g in gs:
            h, w_, cb = g.shape
            idx = oracle.unpack(g.cpu().numpy().reshape(-1, cb), c, 4)
            out.append(oracle.dequantize(idx, 16, Q).reshape(h, w_, c))
        return out
    return oracle.Model(SIDE, SIDE, C, C0, C0, 16, 16, Q, Q, grids(mat.grids0, C0),
                        grids(mat.grids1, C0), [np.asarray(a, np.float64) for a in weights], K,
                        64, 0, 0)


def _f8(mat16, w32):
    ws, q8 = [], []
    for l in range(3):
        s = float(np.abs(w32[l]).max()) / 448.0
        ws.append(s)
        q8.append(torch.from_numpy(w32[l] / s).to(DEV).to(torch.float8_e4m3fn).view(torch.uint8))
    scale = torch.tensor(ws + [1.0 / 256, 16.0 / 256, 16.0 / 256], dtype=torch.float32, device=DEV)
    # FP8 operands take K in steps of 32: W1 padded with zero columns to 64
    q8[0] = torch.nn.functional.pad(q8[0], (0, 64 - K))
    return mat16.with_(weights=q8, precision=ntc.PREC_F8, scale=scale, k_in=64)


def test_render_precision_sweep(trained):
    tr = trained
    m16 = tr.export(ntc.PREC_F16)
    m32 = tr.export(ntc.PREC_F32)
    w32 = [x.cpu().numpy() for x in tr.w_master]
    b32 = [x.cpu().numpy() for x in tr.b]
    m8 = _f8(m16, w32)
    q = gen.camera_queries(320, 180, SIDE, oracle.mips(SIDE, SIDE))
    uvl = torch.from_numpy(q).to(DEV)
    ref = _oracle_model(m32, [w32[0], b32[0], w32[1], b32[1], w32[2], b32[2]]).decode_trilinear(q)
    got = {}
    for name, m in (("f32", m32), ("f16", m16), ("f8", m8)):
        got[name] = to_np(ntc.ntc_decode(m, uvl, filter=ntc.FILTER_TRILINEAR))
        assert ntc.ntc_device_status() == ntc.OK
    p = {k: oracle.psnr(ref, v) for k, v in got.items()}
    assert np.abs(got["f32"] - ref).max() < 1e-4
    assert p["f32"] > 90.0 and p["f16"] > 55.0 and p["f8"] > 30.0, p
    assert p["f32"] > p["f16"] > p["f8"], p
    # stored-weight parity of the FP16 form
    w16 = [x.float().cpu().numpy() for x in m16.weights]
    ref16 = _oracle_model(m16, [w16[0], b32[0], w16[1], b32[1], w16[2], b32[2]]).decode_trilinear(q)
    assert np.abs(got["f16"] - ref16).max() <= 2e-3


def test_export_is_the_quantised_training_state(trained):
    """Exported indices equal the oracle's quantiser applied to the trained
    FP32 grid values (bit-exact)."""
    m16 = trained.export(ntc.PREC_F16)
    for g32, gp in zip(trained.material.grids0 + trained.material.grids1, m16.grids0 + m16.grids1):
        vals = g32.cpu().numpy().astype(np.float64).reshape(-1, C0)
        want = oracle.quantize(vals, 16, Q)
        got = oracle.unpack(gp.cpu().numpy().reshape(vals.shape[0], -1), C0, 4)
        assert np.array_equal(got, want)
