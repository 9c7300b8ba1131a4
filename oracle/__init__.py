"""Plain CPU FP64 oracle for neural texture compression (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library: the arithmetic lives in
``ntc_oracle.c`` (plain C, double precision) and in the few numpy helpers
below, each citing the paper passage it restates.

Paper: "Random-Access Neural Compression of Material Textures" (2023).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_LEVELS = 8


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (portable flags; no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ntc_oracle.h"))):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        # no FMA contraction: FP32 decisions (stochastic texel choice) are
        # evaluated one operation at a time, as written
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class _Model(C.Structure):
    _fields_ = [
        ("width", C.c_int), ("height", C.c_int), ("channels", C.c_int), ("mips", C.c_int),
        ("levels", C.c_int), ("c0", C.c_int), ("c1", C.c_int), ("n0", C.c_int), ("n1", C.c_int),
        ("q0", C.c_double), ("q1", C.c_double),
        ("g0w", C.c_int * MAX_LEVELS), ("g0h", C.c_int * MAX_LEVELS),
        ("g1w", C.c_int * MAX_LEVELS), ("g1h", C.c_int * MAX_LEVELS),
        ("grid0", C.c_void_p * MAX_LEVELS), ("grid1", C.c_void_p * MAX_LEVELS),
        ("k_in", C.c_int), ("hidden", C.c_int), ("act", C.c_int), ("out_act", C.c_int),
        ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
        ("w3", C.c_void_p), ("b3", C.c_void_p), ("interp0", C.c_int),
        ("hidden_layers", C.c_int), ("wm", C.c_void_p), ("bm", C.c_void_p),
        ("vq_g0", C.c_int), ("f8_sa", C.c_void_p),
    ]


class _Noise(C.Structure):
    _fields_ = [("enabled", C.c_int), ("seed", C.c_uint64), ("step", C.c_int64)]


class _Grads(C.Structure):
    _fields_ = [("grid0", C.c_void_p * MAX_LEVELS), ("grid1", C.c_void_p * MAX_LEVELS),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p),
                ("b2", C.c_void_p), ("w3", C.c_void_p), ("b3", C.c_void_p),
                ("wm", C.c_void_p), ("bm", C.c_void_p), ("rows", C.c_void_p)]


_P, _I, _I64, _U64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
# name -> (restype, argtypes) of every function of ntc_oracle.h
SIGNATURES = {
    "or_mips": (_I, [_I, _I]),
    "or_pyramid": (_I, [_I, _I, _P, _P, _P, _P]),
    "or_level_of_mip": (_I, [_I, _I]),
    "or_quantize": (None, [_P, _I64, _I, _D, _P]),
    "or_dequantize": (None, [_P, _I64, _I, _D, _P]),
    "or_cell_bytes": (_I, [_I, _I]),
    "or_pack": (None, [_P, _I64, _I, _I, _P]),
    "or_unpack": (None, [_P, _I64, _I, _I, _P]),
    "or_splitmix64": (_U64, [_U64]),
    "or_rng": (_U64, [_U64, _U64, _U64]),
    "or_noise_value": (_D, [_U64, _I64, _I, _I, _I64, _I, _I, _D]),
    "or_sample_batch": (None, [_U64, _I64, _I64, _I, _I, _I, _P]),
    "or_sample_batch_crops": (None, [_U64, _I64, _I64, _I, _I, _I, _P]),
    "or_positional_encoding": (None, [_I, _I, _P]),
    "or_activation": (_D, [_I, _D]),
    "or_activation_grad": (_D, [_I, _D]),
    "or_features": (None, [_P, _I, _I, _I, _P, _P]),
    "or_features_uvl": (None, [_P, _I64, _P, _P]),
    "or_decode_xym": (None, [_P, _I64, _P, _P, _P, _I]),
    "or_decode_uvl": (None, [_P, _I64, _P, _P, _P, _I]),
    "or_decode_trilinear": (None, [_P, _I64, _P, _P, _I]),
    "or_decode_stochastic": (None, [_P, _I64, _P, C.c_uint64, _I64, _P, _I]),
    "or_backward_xym": (None, [_P, _I64, _P, _P, _P, _P, _I]),
    "or_round_e4m3": (_D, [_D]),
    "or_loss_grad_xym": (_D, [_P, _I64, _P, _P, _P, _P, _I]),
    "or_cosine_lr": (_D, [_D, _I64, _I64]),
    "or_adam": (None, [_P, _P, _P, _P, _I64, _D, _I64, _D, _D, _D, _I, _D, _D]),
}


def _declare(L):
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# pyramid / quantisation helpers
# ---------------------------------------------------------------------------
def mips(width: int, height: int) -> int:
    return lib().or_mips(width, height)


def pyramid(width: int, height: int):
    """Feature-level grid sizes (Sec. 4.1, Table 1): list of
    ``((g0w, g0h), (g1w, g1h))`` per level."""
    a = [np.zeros(MAX_LEVELS, np.int32) for _ in range(4)]
    n = lib().or_pyramid(width, height, *[_p(x) for x in a])
    return [((int(a[0][j]), int(a[1][j])), (int(a[2][j]), int(a[3][j]))) for j in range(n)]


def level_of_mip(m: int, levels: int) -> int:
    return lib().or_level_of_mip(m, levels)


def quantize(x: np.ndarray, n_levels: int, q: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.shape, np.int32)
    lib().or_quantize(_p(x), x.size, n_levels, q, _p(out))
    return out


def dequantize(idx: np.ndarray, n_levels: int, q: float) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.shape, np.float64)
    lib().or_dequantize(_p(idx), idx.size, n_levels, q, _p(out))
    return out


def cell_bytes(c: int, bits: int) -> int:
    return lib().or_cell_bytes(c, bits)


def pack(idx: np.ndarray, c: int, bits: int) -> np.ndarray:
    """Pack ``[cells, c]`` indices into ``[cells, cell_bytes]`` uint8."""
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, c)
    cb = cell_bytes(c, bits)
    out = np.empty((idx.shape[0], cb), np.uint8)
    lib().or_pack(_p(idx), idx.shape[0], c, bits, _p(out))
    return out


def unpack(packed: np.ndarray, c: int, bits: int) -> np.ndarray:
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    cb = cell_bytes(c, bits)
    cells = packed.size // cb
    out = np.empty((cells, c), np.int32)
    lib().or_unpack(_p(packed), cells, c, bits, _p(out))
    return out


def quant_range(n_levels: int, q: float):
    """Continuous clamp range [-(N-1)/2 Q, N/2 Q] (Sec. 4.2)."""
    return -(n_levels - 1) / 2.0 * q, n_levels / 2.0 * q


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------
def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x))


def rng(seed: int, stream: int, counter: int) -> int:
    return int(lib().or_rng(seed, stream, counter))


def noise_value(seed, step, level, grid, cell, ch, c, q) -> float:
    return float(lib().or_noise_value(seed, step, level, grid, cell, ch, c, q))


def sample_batch(seed: int, step: int, batch: int, width: int, height: int, n_mips: int,
                 crops: bool = False):
    """``[batch, 3]`` int32 rows (x, y, m) of one training batch (Sec. 5.1):
    independent texels, or 256 x 256 crops of one mip when ``crops``."""
    out = np.empty((batch, 3), np.int32)
    fn = lib().or_sample_batch_crops if crops else lib().or_sample_batch
    fn(seed, step, batch, width, height, n_mips, _p(out))
    return out


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest FP8-E4M3 value, ties to even, saturating at
    +-448: the OCP 8-bit floating-point format with 1 sign bit, 4 exponent
    bits (bias 7) and 3 mantissa bits, no infinities; binade [2^e, 2^(e+1))
    holds multiples of 2^(e-3) for e >= -6, below 2^-6 the subnormals are
    multiples of 2^-9."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                           # a = f 2^e, f in [0.5, 1)
    quantum = np.ldexp(1.0, np.maximum(e - 1, -6) - 3)
    r = np.minimum(np.rint(a / quantum) * quantum, 448.0)   # rint: half to even
    return np.copysign(r, x)


def vq_reconstruct(idx: np.ndarray, codebooks: np.ndarray) -> np.ndarray:
    """Vector-quantised grid (the paper's comparison with vector
    quantisation): every cell of ``idx`` ``[..., books]`` (uint8) maps to the
    sum over b of entry idx[..., b] of codebook b (``[books, 256, c]``);
    float64 ``[..., c]``."""
    idx = np.asarray(idx)
    cb = np.asarray(codebooks, np.float64)
    out = np.zeros(idx.shape[:-1] + (cb.shape[2],), np.float64)
    for b in range(cb.shape[0]):
        out += cb[b][idx[..., b].astype(np.int64)]
    return out


def vq_assign(values: np.ndarray, codebooks: np.ndarray) -> np.ndarray:
    """Greedy residual vector quantisation of rows ``values`` ``[n, c]``:
    index b is the entry of codebook b nearest to what books 0..b-1 leave of
    the row (squared distance in FP32, channels summed in order, ties to the
    lowest index), then the entry is subtracted.  uint8 ``[n, books]``."""
    r = np.array(values, np.float32)
    cb = np.asarray(codebooks, np.float32)
    n, c = r.shape
    idx = np.zeros((n, cb.shape[0]), np.uint8)
    for b in range(cb.shape[0]):
        best = np.full(n, np.inf, np.float32)
        kb = np.zeros(n, np.int64)
        for k in range(256):
            d = np.zeros(n, np.float32)
            for ch in range(c):
                df = (r[:, ch] - cb[b, k, ch]).astype(np.float32)
                d = (d + (df * df).astype(np.float32)).astype(np.float32)
            better = d < best
            best[better] = d[better]
            kb[better] = k
        idx[:, b] = kb
        r = (r - cb[b][kb]).astype(np.float32)
    return idx


def vq_train_terms(z_levels, codebooks, beta: float):
    """The vector-quantisation terms of one training step of a
    vector-quantised G0 (VQ-VAE, van den Oord et al. 2017, as the paper's
    comparison cites): per level, indices of the latent rows z by greedy
    residual search (``vq_assign``), q = the sum of the selected entries;
    codebook loss (1/N) sum_cells sum_b ||r_b - e_b||^2 with the residuals
    r_b held fixed, and commitment loss beta (1/N) sum ||z - q||^2 with q
    held fixed, N = every G0 latent value.  Returns (indices, q, dL/dz of the
    commitment term, dL/dcodebooks of the codebook term) per level / total,
    float64."""
    cb32 = np.asarray(codebooks, np.float32)
    cb = cb32.astype(np.float64)
    n = sum(np.asarray(z).size for z in z_levels)
    idx_l, q_l, dz_l = [], [], []
    d_cb = np.zeros_like(cb)
    for z in z_levels:
        zf = np.asarray(z, np.float32).reshape(-1, cb.shape[2])
        idx = vq_assign(zf, cb32)
        r = zf.astype(np.float64)
        for b in range(cb.shape[0]):
            e = cb[b][idx[:, b].astype(np.int64)]
            np.add.at(d_cb[b], idx[:, b].astype(np.int64), 2.0 / n * (e - r))
            r = r - e
        q = vq_reconstruct(idx, cb32)
        idx_l.append(idx.reshape(np.asarray(z).shape[:-1] + (cb.shape[0],)))
        q_l.append(q.reshape(np.asarray(z).shape))
        dz_l.append((2.0 * beta / n * (zf.astype(np.float64) - q)).reshape(np.asarray(z).shape))
    return idx_l, q_l, dz_l, d_cb


def activation(act: int, z: float) -> float:
    return float(lib().or_activation(act, z))


def activation_grad(act: int, z: float) -> float:
    return float(lib().or_activation_grad(act, z))


def positional_encoding(x: int, y: int) -> np.ndarray:
    out = np.empty(12, np.float64)
    lib().or_positional_encoding(x, y, _p(out))
    return out


# ---------------------------------------------------------------------------
# model
# ---------------------------------------------------------------------------
class Model:
    """One material: latent grids (float64 values) + decoder weights.

    ``grids0[j]`` is ``[g0h, g0w, c0]``, ``grids1[j]`` ``[g1h, g1w, c1]``;
    ``weights`` is ``[w1, b1, w2, b2, w3, b3]`` (two hidden layers) or
    ``[w1, b1, w2, b2, wm, bm, w3, b3]`` (three: the third hidden layer wm
    before the output layer w3), layer order, ``w`` stored ``[out][in]``.  ``act`` 0 = ReLU, 1 = hardGELU; ``out_act`` 0 = sigmoid,
    1 = identity.
    """

    def __init__(self, width, height, channels, c0, c1, n0, n1, q0, q1, grids0, grids1,
                 weights, k_in, hidden=64, act=0, out_act=0, interp0=0, vq_g0=False):
        self.width, self.height, self.channels = width, height, channels
        self.mips = mips(width, height)
        self.levels = len(grids0)
        self.c0, self.c1, self.n0, self.n1, self.q0, self.q1 = c0, c1, n0, n1, q0, q1
        self.grids0 = [np.ascontiguousarray(g, np.float64) for g in grids0]
        self.grids1 = [np.ascontiguousarray(g, np.float64) for g in grids1]
        self.weights = [np.ascontiguousarray(w, np.float64) for w in weights]
        self.k_in, self.hidden, self.act, self.out_act = k_in, hidden, act, out_act
        s = _Model()
        s.width, s.height, s.channels, s.mips, s.levels = width, height, channels, self.mips, self.levels
        s.c0, s.c1, s.n0, s.n1, s.q0, s.q1 = c0, c1, n0, n1, q0, q1
        for j in range(self.levels):
            s.g0h[j], s.g0w[j] = self.grids0[j].shape[:2]
            s.g1h[j], s.g1w[j] = self.grids1[j].shape[:2]
            s.grid0[j] = self.grids0[j].ctypes.data
            s.grid1[j] = self.grids1[j].ctypes.data
        s.k_in, s.hidden, s.act, s.out_act = k_in, hidden, act, out_act
        self.interp0 = s.interp0 = interp0
        self.vq_g0 = s.vq_g0 = int(bool(vq_g0))
        w = self.weights
        assert len(w) in (6, 8)
        self.hidden_layers = s.hidden_layers = 2 if len(w) == 6 else 3
        s.w1, s.b1, s.w2, s.b2 = [a.ctypes.data for a in w[:4]]
        s.w3, s.b3 = w[-2].ctypes.data, w[-1].ctypes.data
        if len(w) == 8:
            s.wm, s.bm = w[4].ctypes.data, w[5].ctypes.data
            assert w[4].shape == (hidden, hidden)
        assert w[0].shape == (hidden, k_in) and w[2].shape == (hidden, hidden)
        assert w[-2].shape == (channels, hidden)
        self._s = s

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _noise(noise):
        if noise is None:
            return None, None
        n = _Noise(1, noise[0], noise[1])
        return n, C.byref(n)

    def features(self, x, y, m, noise=None):
        row = np.empty(self.k_in, np.float64)
        _, nz = self._noise(noise)
        lib().or_features(C.byref(self._s), x, y, m, nz, _p(row))
        return row

    def features_uvl(self, uvl):
        """``[n, k_in]`` MLP input rows of the nearest texels of ``uvl``."""
        uvl = np.ascontiguousarray(uvl, np.float32).reshape(-1, 3)
        rows = np.empty((uvl.shape[0], self.k_in), np.float64)
        lib().or_features_uvl(C.byref(self._s), uvl.shape[0], _p(uvl), _p(rows))
        return rows

    def decode_f8(self, uvl, s_w, s_a):
        """Nearest decode in the FP8-E4M3 precision form: layer l computes
        (s_w[l] s_a[l]) (W_l / s_w[l]) . e4m3(x_l / s_a[l]) + b_l, i.e. the
        stored weights are this model's weights (already E4M3 values times
        s_w[l]) and every layer input is rounded to E4M3 in units of its
        activation scale; everything else in FP64."""
        assert self.hidden_layers == 2, "the FP8 form has two hidden layers"
        w = self.weights
        x = self.features_uvl(uvl)
        for l in range(3):
            a = round_e4m3(x / s_a[l])
            x = (s_w[l] * s_a[l]) * (a @ (w[2 * l] / s_w[l]).T) + w[2 * l + 1]
            if l < 2:
                x = np.vectorize(lambda v: activation(self.act, v))(x)
        if self.out_act == 0:
            x = 1.0 / (1.0 + np.exp(-x))
        return x

    def f8_form(self, s_w, s_a):
        """The FP8-E4M3 training and decode form of this model (the paper
        trains with half-precision tensor cores, Sec. 5.1, and leaves lower
        precision to future work, Sec. 7): every weight
        matrix replaced by s_w[l] e4m3(W_l / s_w[l]) (biases unchanged) and
        every layer input used as s_a[l] e4m3(v / s_a[l]) inside the C
        forward.  Its reverse mode is straight-through: each rounding counts
        as the identity, the weight gradients use the rounded inputs, and the
        returned weight gradients are those of the quantised weights (which a
        trainer applies to its master weights).  Two hidden layers."""
        assert self.hidden_layers == 2, "the FP8 form has two hidden layers"
        w = list(self.weights)
        for l in range(3):
            w[2 * l] = s_w[l] * np.vectorize(lib().or_round_e4m3)(w[2 * l] / s_w[l])
        f8 = Model(self.width, self.height, self.channels, self.c0, self.c1, self.n0, self.n1,
                   self.q0, self.q1, self.grids0, self.grids1, w, self.k_in, self.hidden,
                   self.act, self.out_act, self.interp0, bool(self.vq_g0))
        f8._sa = np.ascontiguousarray(s_a, np.float64).reshape(3)
        f8._s.f8_sa = f8._sa.ctypes.data
        return f8

    def decode_xym(self, xym, noise=None, threads=None):
        xym = np.ascontiguousarray(xym, np.int32).reshape(-1, 3)
        out = np.empty((xym.shape[0], self.channels), np.float64)
        _, nz = self._noise(noise)
        lib().or_decode_xym(C.byref(self._s), xym.shape[0], _p(xym), nz, _p(out),
                            threads or default_threads())
        return out

    def decode(self, uvl, noise=None, threads=None):
        """Nearest-texel decode of ``[n, 3]`` float32 (u, v, lod) queries."""
        uvl = np.ascontiguousarray(uvl, np.float32).reshape(-1, 3)
        out = np.empty((uvl.shape[0], self.channels), np.float64)
        _, nz = self._noise(noise)
        lib().or_decode_uvl(C.byref(self._s), uvl.shape[0], _p(uvl), nz, _p(out),
                            threads or default_threads())
        return out

    def decode_trilinear(self, uvl, threads=None):
        uvl = np.ascontiguousarray(uvl, np.float32).reshape(-1, 3)
        out = np.empty((uvl.shape[0], self.channels), np.float64)
        lib().or_decode_trilinear(C.byref(self._s), uvl.shape[0], _p(uvl), _p(out),
                                  threads or default_threads())
        return out

    def decode_stochastic(self, uvl, seed, step, threads=None):
        """Stochastic filtering (Sec. 5.3) of frame `step`: one jittered nearest
        decode per query."""
        uvl = np.ascontiguousarray(uvl, np.float32).reshape(-1, 3)
        out = np.empty((uvl.shape[0], self.channels), np.float64)
        lib().or_decode_stochastic(C.byref(self._s), uvl.shape[0], _p(uvl), seed, step, _p(out),
                                   threads or default_threads())
        return out

    def zero_grads(self, n_rows=None):
        g = {"grid0": [np.zeros_like(a) for a in self.grids0],
             "grid1": [np.zeros_like(a) for a in self.grids1],
             "w": [np.zeros_like(a) for a in self.weights]}
        s = _Grads()
        if n_rows is not None:
            g["rows"] = np.zeros((n_rows, self.k_in), np.float64)
            s.rows = g["rows"].ctypes.data
        for j in range(self.levels):
            s.grid0[j] = g["grid0"][j].ctypes.data
            s.grid1[j] = g["grid1"][j].ctypes.data
        gw = g["w"]
        s.w1, s.b1, s.w2, s.b2 = [a.ctypes.data for a in gw[:4]]
        s.w3, s.b3 = gw[-2].ctypes.data, gw[-1].ctypes.data
        if len(gw) == 8:
            s.wm, s.bm = gw[4].ctypes.data, gw[5].ctypes.data
        g["_s"] = s
        return g

    def backward_xym(self, xym, dout, noise=None, threads=None, rows=False):
        """Gradients of sum(dout * y) (exact reverse mode; straight-through
        in the FP8 form); ``rows``: also each texel's input-row gradient
        (``g["rows"]``, ``[n, k_in]``)."""
        xym = np.ascontiguousarray(xym, np.int32).reshape(-1, 3)
        dout = np.ascontiguousarray(dout, np.float64).reshape(xym.shape[0], self.channels)
        g = self.zero_grads(xym.shape[0] if rows else None)
        _, nz = self._noise(noise)
        lib().or_backward_xym(C.byref(self._s), xym.shape[0], _p(xym), _p(dout), nz,
                              C.byref(g["_s"]), threads or default_threads())
        return g

    def loss_grad_xym(self, xym, target, noise=None, threads=None, rows=False):
        """L2 loss (Sec. 4.5) and its gradients for texels ``xym`` with
        ``target`` ``[n, c]`` in [0, 1]."""
        xym = np.ascontiguousarray(xym, np.int32).reshape(-1, 3)
        target = np.ascontiguousarray(target, np.float64).reshape(xym.shape[0], self.channels)
        g = self.zero_grads(xym.shape[0] if rows else None)
        _, nz = self._noise(noise)
        loss = lib().or_loss_grad_xym(C.byref(self._s), xym.shape[0], _p(xym), _p(target), nz,
                                      C.byref(g["_s"]), threads or default_threads())
        return float(loss), g


def uvl_of_xym(xym: np.ndarray, width: int, height: int) -> np.ndarray:
    """Texel-centre (u, v, lod) query rows for integer texels (x, y, m)."""
    xym = np.asarray(xym).reshape(-1, 3)
    m = xym[:, 2].astype(np.int64)
    wm = np.maximum(1, width >> m)
    hm = np.maximum(1, height >> m)
    out = np.empty((xym.shape[0], 3), np.float32)
    out[:, 0] = (xym[:, 0] + 0.5) / wm
    out[:, 1] = (xym[:, 1] + 0.5) / hm
    out[:, 2] = m
    return out


def targets_of_xym(mip_chain_u8, xym) -> np.ndarray:
    """Reference values t = q/255 of 8-bit mip texels (App. I: 8-bit sources)."""
    xym = np.asarray(xym).reshape(-1, 3)
    c = mip_chain_u8[0].shape[2]
    out = np.empty((xym.shape[0], c), np.float64)
    for m in np.unique(xym[:, 2]):
        sel = xym[:, 2] == m
        lvl = mip_chain_u8[int(m)]
        out[sel] = lvl[xym[sel, 1], xym[sel, 0]].astype(np.float64) / 255.0
    return out


def cosine_lr(lr0: float, t: int, total: int) -> float:
    return float(lib().or_cosine_lr(lr0, t, total))


def adam(p, m, v, g, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, clamp=None):
    """In-place FP64 Adam step on contiguous float64 arrays."""
    lo, hi = clamp if clamp is not None else (0.0, 0.0)
    lib().or_adam(_p(p), _p(m), _p(v), _p(np.ascontiguousarray(g, np.float64)), p.size, lr, t,
                  beta1, beta2, eps, 1 if clamp is not None else 0, lo, hi)


# ---------------------------------------------------------------------------
# metrics and storage (numpy)
# ---------------------------------------------------------------------------
def texture_set_psnr(ref_levels, test_levels) -> float:
    """Texture-set PSNR over a mip chain (App. H, Eq. 1): the squared error
    summed over every mip and channel, divided by c * sum_j w_j h_j, peak 1."""
    se, count = 0.0, 0
    for r, t in zip(ref_levels, test_levels):
        d = np.asarray(r, np.float64) - np.asarray(t, np.float64)
        se += float(np.sum(d * d))
        count += d.size
    mse = se / count
    return float("inf") if mse == 0.0 else -10.0 * math.log10(mse)


def psnr(ref, test) -> float:
    """PSNR of two equally shaped arrays with values in [0, 1]."""
    return texture_set_psnr([ref], [test])


def grid_storage_bytes(width: int, height: int, c0: int, b0: int, c1: int, b1: int,
                       all_levels: bool = True, g0_side: int | None = None) -> float:
    """Bytes of the quantised feature pyramid (App. E, Table 5): c*B bits per
    cell, densely packed, summed over every feature level's two grids (or
    over level 0 only).  ``g0_side`` overrides the level-0 G0 side (W/4 in
    Table 1; profiles 1.0 and 2.25 use W/2); later levels shrink by 4."""
    if g0_side is None:
        levels = pyramid(width, height)
    else:
        levels = pyramid(4 * g0_side, 4 * g0_side * height // width)
    if not all_levels:
        levels = levels[:1]
    bits = 0
    for (g0w, g0h), (g1w, g1h) in levels:
        bits += g0w * g0h * c0 * b0 + g1w * g1h * c1 * b1
    return bits / 8.0


def lod_law_probs(n_mips: int, uniform_frac: float = 0.05) -> np.ndarray:
    """P(m) of the training LOD sampler (Sec. 5.1): floor(-log4 X) has
    P(m) = 3 * 4^-(m+1), the tail folded into the last mip, mixed with a
    uniform choice over all mips at ``uniform_frac``."""
    p = np.array([3.0 * 4.0 ** -(m + 1) for m in range(n_mips)])
    p[-1] = 1.0 - p[:-1].sum()
    return (1.0 - uniform_frac) * p + uniform_frac / n_mips
