"""ntc_decode_host: host query and output buffers, chunks streamed through a
device workspace with the copies overlapping the decode on helper streams.
Outputs must equal ntc_decode's bit for bit (every query is decoded by the
same kernel from the same inputs), for any chunking, also when captured in
a CUDA graph and replayed."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def _ws(mat, chunk, dtype):
    dt = ntc.DTYPE_F16 if dtype == torch.float16 else ntc.DTYPE_F32
    return torch.empty(ntc.lib().ntc_decode_host_workspace_bytes(mat.channels, dt, chunk),
                       dtype=torch.uint8, device=DEV)


@pytest.mark.parametrize("chunk", [128, 1024, 1 << 16])
@pytest.mark.parametrize("dtype", [torch.float16, torch.float32])
@pytest.mark.parametrize("filt", [ntc.FILTER_NEAREST, ntc.FILTER_TRILINEAR])
def test_decode_host_equals_device_decode(filt, dtype, chunk):
    case = make_case(512, 512, 16, 12, 12, k_in=48, seed=91)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = torch.from_numpy(gen.random_queries(7 * 1024 + 77, md.mips, seed=4091)).pin_memory()
    ref = ntc.ntc_decode(mat, q.to(DEV), out_dtype=dtype, filter=filt).cpu()
    out = torch.empty_like(ref).pin_memory()
    ntc.ntc_decode_host(mat, q, out_host=out, filter=filt, workspace=_ws(mat, chunk, dtype))
    torch.cuda.synchronize()
    assert ntc.ntc_device_status() == ntc.OK
    assert torch.equal(out, ref)


def test_decode_host_fp32_form_with_noise():
    case = make_case(256, 256, 8, 8, 8, k_in=32, seed=92)
    mat, md = device_material(case, precision=ntc.PREC_F32, packed=False)
    q = torch.from_numpy(gen.random_queries(3000, md.mips, seed=4092)).pin_memory()
    kw = dict(flags=ntc.FLAG_NOISE, noise_seed=5, noise_step=2)
    ref = ntc.ntc_decode(mat, q.to(DEV), **kw).cpu()
    out = ntc.ntc_decode_host(mat, q, workspace=_ws(mat, 256, torch.float32), **kw)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_decode_host_in_a_cuda_graph():
    case = make_case(512, 512, 16, 12, 12, k_in=48, seed=93)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = torch.from_numpy(gen.random_queries(5000, md.mips, seed=4093)).pin_memory()
    out = torch.zeros((5000, 16), dtype=torch.float16).pin_memory()
    ws = _ws(mat, 1024, torch.float16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up outside capture (helper streams created)
        ntc.ntc_decode_host(mat, q, out_host=out, workspace=ws, stream=s)
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ntc.ntc_decode_host(mat, q, out_host=out, workspace=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    ref = ntc.ntc_decode(mat, q.to(DEV), out_dtype=torch.float16).cpu()
    assert torch.equal(out, ref)
