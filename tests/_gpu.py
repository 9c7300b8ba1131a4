"""Device-side construction of the seeded cases for the GPU parity tests.

Packed grids are produced by the oracle's packer from the case's indices (an
input encoding, identical for both sides); the library's own packer is
checked bit-exactly against it separately.
"""
import numpy as np
import torch

import oracle
import paper_2305_17105_gb300 as ntc

DEV = "cuda"


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def stored_weights(case, precision):
    """The weights as the library stores them (layer order, 3 or 4 layers)
    and the exactly converted float64 values the oracle then sees
    (stored-weight parity)."""
    w = case.weights
    oracle_w = []
    dev = []
    for l in range(len(w) // 2):
        wl = w[2 * l].astype(np.float16) if precision == ntc.PREC_F16 else w[2 * l]
        dev.append(_t(wl))
        oracle_w += [wl.astype(np.float64), w[2 * l + 1]]
    return dev, [np.asarray(x, np.float64) for x in oracle_w]


def device_material(case, precision=ntc.PREC_F32, packed=True):
    """(ntc.Material, oracle.Model) for one case."""
    wdev, wor = stored_weights(case, precision)
    if packed:
        g0 = [_t(oracle.pack(i.reshape(-1, case.c0), case.c0, case.bits0).reshape(
            i.shape[0], i.shape[1], -1)) for i in case.idx0]
        g1 = [_t(oracle.pack(i.reshape(-1, case.c1), case.c1, case.bits1).reshape(
            i.shape[0], i.shape[1], -1)) for i in case.idx1]
    else:
        g0 = [_t(v) for v in case.val0]
        g1 = [_t(v) for v in case.val1]
    b = [_t(x) for x in case.weights[1::2]]
    mat = ntc.Material(case.width, case.height, case.channels, case.c0, case.c1, case.bits0,
                       case.bits1, case.q0, case.q1, g0, g1, wdev, b, case.k_in, precision,
                       case.act, case.out_act, interp0=case.interp0)
    md = case.oracle_model(weights=wor, quantized=packed)
    return mat, md


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def rel_err(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


# Gradient bar: 1e-2 relative error (L2 norm) per tensor, for the FP32 form
# and for the FP16 tensor-core form.  The FP16 form meets it because its
# forward feeds each ReLU / hardGELU layer an FP16 head plus an FP16 tail of
# its input (the activation masks are then those of the exact forward); its
# backward products stay plain FP16 with FP32 accumulation (~3e-4).
def check_grads(got_views, refs, n_grids, fp16):
    got = [np.asarray(to_np(v), np.float64).reshape(-1) for v in got_views]
    ref = [np.asarray(r, np.float64).reshape(-1) for r in refs]
    errs = [rel_err(g, r) for g, r in zip(got, ref)]
    for k, err in enumerate(errs):
        assert err <= 1e-2, (k, err, errs)
    return errs
