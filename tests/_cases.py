"""Seeded material cases shared by the oracle tests and the GPU parity tests.

A case holds plain numpy inputs (grid values or grid indices, MLP weights,
queries); the oracle and the CUDA library each receive them and compute on
their own.  Grid shapes come from the oracle's pyramid rule (Table 1); the GPU
tests check separately that the library's own rule agrees.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import ntc_inputs as gen
import oracle


@dataclasses.dataclass
class Case:
    width: int
    height: int
    channels: int
    c0: int
    c1: int
    bits0: int
    bits1: int
    q0: float
    q1: float
    k_in: int
    hidden: int
    act: int
    out_act: int
    levels: list            # [((g0w, g0h), (g1w, g1h))]
    idx0: list              # per level [g0h, g0w, c0] int32 indices (packed form)
    idx1: list
    val0: list              # per level float32 values
    val1: list
    weights: list           # [w1, b1, w2, b2, (wm, bm,) w3, b3] float32, layer order
    interp0: int = 0        # G0 resampling: 0 bilinear, 1 learned (4 taps concatenated)

    @property
    def hidden_layers(self):
        return len(self.weights) // 2 - 1

    @property
    def mips(self):
        return oracle.mips(self.width, self.height)

    @property
    def n0(self):
        return 1 << self.bits0

    @property
    def n1(self):
        return 1 << self.bits1

    def oracle_model(self, weights=None, quantized=True):
        """The oracle's model: dequantised indices (packed form) or the raw
        float values (training form)."""
        if quantized:
            g0 = [oracle.dequantize(i, self.n0, self.q0) for i in self.idx0]
            g1 = [oracle.dequantize(i, self.n1, self.q1) for i in self.idx1]
        else:
            g0 = [v.astype(np.float64) for v in self.val0]
            g1 = [v.astype(np.float64) for v in self.val1]
        w = self.weights if weights is None else weights
        return oracle.Model(self.width, self.height, self.channels, self.c0, self.c1, self.n0,
                            self.n1, self.q0, self.q1, g0, g1, [np.asarray(a, np.float64) for a in w],
                            self.k_in, self.hidden, self.act, self.out_act, self.interp0)


def make_case(width=64, height=64, channels=8, c0=8, c1=8, bits0=4, bits1=4, q0=None, q1=None,
              k_in=None, hidden=64, act=0, out_act=0, seed=0, wgain=1.0, interp0=0,
              hidden_layers=2):
    n0, n1 = 1 << bits0, 1 << bits1
    q0 = 1.0 / n0 if q0 is None else q0
    q1 = 1.0 / n1 if q1 is None else q1
    used = (4 * c0 if interp0 else c0) + c1 + 13
    if k_in is None:
        k_in = (used + 15) // 16 * 16
    rng = np.random.default_rng(1000 + seed)
    levels = oracle.pyramid(width, height)
    idx0, idx1, val0, val1 = [], [], [], []
    lo0, hi0 = oracle.quant_range(n0, q0)
    lo1, hi1 = oracle.quant_range(n1, q1)
    for (g0w, g0h), (g1w, g1h) in levels:
        idx0.append(rng.integers(0, n0, size=(g0h, g0w, c0)).astype(np.int32))
        idx1.append(rng.integers(0, n1, size=(g1h, g1w, c1)).astype(np.int32))
        val0.append(gen.uniform_grid_values((g0h, g0w, c0), lo0, hi0, rng))
        val1.append(gen.uniform_grid_values((g1h, g1w, c1), lo1, hi1, rng))
    weights = gen.random_mlp(k_in, hidden, channels, 2000 + seed, n_used=used, gain=wgain,
                             hidden_layers=hidden_layers)
    return Case(width, height, channels, c0, c1, bits0, bits1, q0, q1, k_in, hidden, act, out_act,
                levels, idx0, idx1, val0, val1, weights, interp0)


# The five workload shapes (sizes of the paper-shaped synthetic workloads).
def case_small_fp32(seed=0):
    """256^2 x 8 material; G0 64^2 x 8, G1 32^2 x 8, 4-bit features uniform in
    [-1, 1] (bin width 2/16); K = 32; hidden 64; 8 sigmoid outputs."""
    return make_case(256, 256, 8, 8, 8, 4, 4, q0=2.0 / 16, q1=2.0 / 16, k_in=32, seed=seed)


def case_decode_4k(seed=0):
    """4096^2 x 16 material, 13 mips; G0 1024^2 x 12, G1 512^2 x 12, 4 bits;
    MLP 48 -> 64 -> 64 -> 16."""
    return make_case(4096, 4096, 16, 12, 12, 4, 4, k_in=48, seed=seed)


def case_train_2k(seed=0):
    """2048^2 x 12 material; G0 512^2 x 16, G1 256^2 x 16 (4-bit range);
    MLP 48 -> 64 -> 64 -> 12."""
    return make_case(2048, 2048, 12, 16, 16, 4, 4, k_in=48, seed=seed)
