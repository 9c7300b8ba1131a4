"""Many materials in one persistent launch: parity with the single-material
decode (same arithmetic) and with the FP64 oracle, CUDA-graph capture of the
batched decode and of a multi-material training loop."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import oracle
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material, rel_err, to_np

pytestmark = pytest.mark.gpu
OUT_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _uvl(q):
    return torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(DEV)


def _materials(shapes, seed, **kw):
    out = []
    for i, (side, c) in enumerate(shapes):
        case = make_case(side, side, c, 12, 12, k_in=48, seed=seed + i, **kw)
        out.append(device_material(case, precision=ntc.PREC_F16))
    return out


@pytest.mark.parametrize("filt", [ntc.FILTER_NEAREST, ntc.FILTER_TRILINEAR])
def test_batched_decode_matches_single_and_oracle(filt):
    shapes = [(256, 8), (64, 12), (512, 16), (128, 16), (256, 12), (32, 8)]
    mats = _materials(shapes, seed=80)
    nq = [1000, 0, 3 * 128 + 5, 1, 129, 700]
    qs = [gen.random_queries(n, oracle.mips(s, s), seed=4080 + i) for i, ((s, _), n) in
          enumerate(zip(shapes, nq))]
    if filt == ntc.FILTER_TRILINEAR:
        for q in qs:
            q[:, 2] += np.float32(0.37)
    batch = ntc.Batch([m for m, _ in mats], nq, filter=filt)
    uvl = _uvl(np.concatenate(qs))
    out = to_np(ntc.ntc_decode_batched(batch, uvl))
    assert ntc.ntc_device_status() == ntc.OK
    for i, ((m, md), q) in enumerate(zip(mats, qs)):
        got = out[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(q), m.channels)
        if len(q) == 0:
            continue
        single = to_np(ntc.ntc_decode(m, _uvl(q), filter=filt))
        assert np.abs(got - single).max() <= 1e-6, i
        ref = md.decode_trilinear(q) if filt == ntc.FILTER_TRILINEAR else md.decode(q)
        assert np.abs(got - ref).max() <= OUT_TOL, i


def test_batched_decode_generic_layout_and_f16_out():
    shapes = [(128, 8), (64, 5)]
    mats = []
    for i, (side, c) in enumerate(shapes):
        case = make_case(side, side, c, 6, 10, bits0=2, bits1=8, k_in=32, seed=90 + i)
        mats.append(device_material(case, precision=ntc.PREC_F16))
    nq = [777, 300]
    qs = [gen.random_queries(n, oracle.mips(s, s), seed=4090 + i) for i, ((s, _), n) in
          enumerate(zip(shapes, nq))]
    batch = ntc.Batch([m for m, _ in mats], nq)
    out = to_np(ntc.ntc_decode_batched(batch, _uvl(np.concatenate(qs)), out_dtype=torch.float16))
    for i, ((m, md), q) in enumerate(zip(mats, qs)):
        got = out[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(q), m.channels)
        assert np.abs(got - md.decode(q)).max() <= OUT_TOL


def test_batched_decode_in_cuda_graph():
    shapes = [(256, 16), (128, 8), (512, 12)]
    mats = _materials(shapes, seed=95)
    nq = [5000, 3000, 4000]
    qs = [gen.random_queries(n, oracle.mips(s, s), seed=4095 + i) for i, ((s, _), n) in
          enumerate(zip(shapes, nq))]
    batch = ntc.Batch([m for m, _ in mats], nq)
    uvl = _uvl(np.concatenate(qs))
    out = torch.empty(int(batch.desc.total_outputs), dtype=torch.float32, device=DEV)
    ref = ntc.ntc_decode_batched(batch, uvl).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ntc.ntc_decode_batched(batch, uvl, out=out)  # warm-up (launch attributes) outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        ntc.ntc_decode_batched(batch, uvl, out=out)
    for _ in range(3):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_multi_material_training_loop_in_cuda_graph():
    """Three materials of different sizes and channel counts, one training
    step each per iteration, captured once as a CUDA graph and replayed: the
    device step counters drive the sampler, the noise and the schedule, so
    replays equal eager steps."""
    trainers, targets = [], []
    for i, (side, c) in enumerate([(128, 8), (64, 12), (256, 16)]):
        case = make_case(side, side, c, 16, 16, k_in=48, seed=100 + i)
        w = case.weights
        mk = lambda: ntc.Trainer(side, side, c, 16, 16, 4, 4, case.q0, case.q1, case.val0,
                                 case.val1, [w[0], w[2], w[4]], [w[1], w[3], w[5]], 48,
                                 ntc.PREC_F16, total_steps=20)
        trainers.append((mk(), mk()))
        targets.append(ntc.Target(gen.box_mip_chain_u8(gen.synthetic_texture(side, side, c,
                                                                             seed=1100 + i))))
    eager = [a for a, _ in trainers]
    graphed = [b for _, b in trainers]

    def step(trs):
        for tr, tg in zip(trs, targets):
            ntc.ntc_train_step(tr, tg, 2048, 17)

    step(graphed)  # warm-up outside capture; both sets then take steps 1..4
    step(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step(graphed)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        g.replay()
        step(eager)
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    for a, b in zip(eager, graphed):
        assert int(a.step_t.item()) == int(b.step_t.item()) == 4
        assert abs(a.loss.item() - b.loss.item()) <= 1e-4 * a.loss.item()
        assert rel_err(to_np(b.params), to_np(a.params)) < 1e-3


def test_batched_decode_mixed_fast_classes_and_channels():
    """Materials whose 4-bit cell layouts differ (fast classes decided per
    material inside the launch), odd channel counts and output blocks that
    are not 8-element aligned."""
    specs = [(128, 3, 8, 8), (256, 16, 12, 12), (64, 5, 16, 16), (128, 7, 8, 16), (256, 12, 13, 10)]
    mats, qs = [], []
    for i, (side, c, c0, c1) in enumerate(specs):
        case = make_case(side, side, c, c0, c1, k_in=48, seed=200 + i)
        mats.append(device_material(case, precision=ntc.PREC_F16))
        qs.append(gen.random_queries(131 * (i + 1) + 3, oracle.mips(side, side), seed=4200 + i))
    batch = ntc.Batch([m for m, _ in mats], [len(q) for q in qs])
    for filt in (ntc.FILTER_NEAREST, ntc.FILTER_TRILINEAR):
        if filt == ntc.FILTER_TRILINEAR:
            batch = ntc.Batch([m for m, _ in mats], [len(q) for q in qs], filter=filt)
        out = to_np(ntc.ntc_decode_batched(batch, _uvl(np.concatenate(qs))))
        assert ntc.ntc_device_status() == ntc.OK
        for i, ((m, md), q) in enumerate(zip(mats, qs)):
            got = out[batch.o_offsets[i]:batch.o_offsets[i + 1]].reshape(len(q), m.channels)
            ref = md.decode_trilinear(q) if filt == ntc.FILTER_TRILINEAR else md.decode(q)
            assert np.abs(got - ref).max() <= OUT_TOL, (filt, i)
