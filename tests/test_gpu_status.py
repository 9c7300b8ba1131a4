"""Failure detection without a GPU fault: a bounded device-side wait that
cannot complete gives up after its limit, records NTC_ERR_TIMEOUT in the
status word and returns; the host reads the status, clears it, and the
context keeps decoding correctly."""
import numpy as np
import pytest
import torch

import ntc_inputs as gen
import paper_2305_17105_gb300 as ntc
from _cases import make_case
from _gpu import DEV, device_material, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ntc.lib()


def test_bounded_wait_reports_timeout_and_context_survives():
    assert ntc.ntc_device_status() == ntc.OK            # clean start (and cleared)
    ntc.ntc_selftest_wait(2000)                         # at most ~20 ms of suspended tries
    assert ntc.ntc_device_status(reset=False) == ntc.ERR_TIMEOUT
    assert ntc.ntc_device_status(reset=True) == ntc.ERR_TIMEOUT
    assert ntc.ntc_device_status() == ntc.OK            # cleared
    case = make_case(256, 256, 8, 8, 8, k_in=32, seed=94)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = gen.random_queries(4096, md.mips, seed=4094)
    out = to_np(ntc.ntc_decode(mat, torch.from_numpy(q).to(DEV)))
    assert ntc.ntc_device_status() == ntc.OK
    assert np.abs(out - md.decode(q)).max() <= 2e-3


def test_selftest_limit_validation():
    with pytest.raises(ntc.NTCError):
        ntc.ntc_selftest_wait(0)
    with pytest.raises(ntc.NTCError):
        ntc.ntc_selftest_wait((1 << 20) + 1)


def test_binding_refuses_short_device_buffers():
    """Buffers shorter than what the library would write (or read) are
    refused by the binding before any launch; the outputs stay untouched."""
    case = make_case(64, 64, 8, 8, 8, k_in=32, seed=95)
    mat, md = device_material(case, precision=ntc.PREC_F16)
    q = torch.from_numpy(gen.random_queries(100, md.mips, seed=4095)).to(DEV)
    short = torch.full((799,), 7.0, device=DEV)
    with pytest.raises(ValueError, match="the call uses 800"):
        ntc.ntc_decode(mat, q, out=short)
    with pytest.raises(ValueError, match="the call uses 800"):
        ntc.ntc_autotune_decode(mat, q, short)
    with pytest.raises(ValueError, match="the call uses 800"):
        ntc.ntc_backward(mat, q, short, ntc.grads_struct(mat))
    with pytest.raises(ValueError, match=r"\[n, 3\] float32"):
        ntc.ntc_decode(mat, q[:, :2].contiguous())
    with pytest.raises(ValueError, match="contiguous"):
        ntc.ntc_decode(mat, q.t().contiguous().t())
    with pytest.raises(ValueError, match="the call uses"):
        ntc.ntc_quantize_pack(torch.zeros(64, device=DEV), 4, 4, 0.25,
                              packed=torch.zeros(1, dtype=torch.uint8, device=DEV))
    batch = ntc.Batch([mat], [100])
    with pytest.raises(ValueError, match="uvl holds"):
        ntc.ntc_decode_batched(batch, q[:99])
    with pytest.raises(ValueError, match="the call uses 800"):
        ntc.ntc_decode_batched(batch, q, out=short)
    torch.cuda.synchronize()
    assert bool((short == 7.0).all())
    assert ntc.ntc_device_status() == ntc.OK
