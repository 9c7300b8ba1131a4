"""GB300 neural texture compression: Python binding of libntc.so.

Thin argument marshalling over the C ABI declared in ``include/ntc.h`` (same
function names).  PyTorch supplies device memory and streams; every step of
the decode and of the optimisation runs in the library's CUDA kernels.  There
is no CPU path: without the compiled library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libntc.so")

MAX_LEVELS = 8
MAX_MIPS = 16
MAX_CHANNELS = 16
MAX_K = 128
HIDDEN = 64
MAX_FEATURES = 32
MAX_BATCH = 1024
MAX_TRAIN_BATCH = 256
NOALLOC_MAX_PARAMS = 1 << 21

OK, ERR_ARG, ERR_SHAPE, ERR_ALIGN, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT = range(7)
GRID_PACKED, GRID_F32 = 0, 1
PREC_F32, PREC_F16, PREC_F8 = 0, 1, 2
ACT_RELU, ACT_HARDGELU = 0, 1
OUT_SIGMOID, OUT_IDENTITY = 0, 1
FILTER_NEAREST, FILTER_TRILINEAR, FILTER_STOCHASTIC = 0, 1, 2
INTERP_BILINEAR, INTERP_LEARNED = 0, 1
DTYPE_F32, DTYPE_F16, DTYPE_U8 = 0, 1, 2
_OUT_DTYPES = {torch.float32: DTYPE_F32, torch.float16: DTYPE_F16, torch.uint8: DTYPE_U8}
FLAG_NOISE, FLAG_FREEZE_GRIDS, FLAG_NO_NOISE, FLAG_SIMT, FLAG_GRAD_ONLY = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_CROPS = 0x20


class NTCError(RuntimeError):
    def __init__(self, name, code, msg):
        super().__init__(f"{name} failed with status {code}: {msg}")
        self.code = code


# ----------------------------------------------------------------------------
# ctypes mirrors of include/ntc.h
# ----------------------------------------------------------------------------
class ntc_level(C.Structure):
    _fields_ = [("g0_w", C.c_int32), ("g0_h", C.c_int32), ("g1_w", C.c_int32), ("g1_h", C.c_int32),
                ("grid0", C.c_void_p), ("grid1", C.c_void_p)]


class ntc_material(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("channels", C.c_int32),
                ("mips", C.c_int32), ("levels", C.c_int32), ("c0", C.c_int32), ("c1", C.c_int32),
                ("bits0", C.c_int32), ("bits1", C.c_int32), ("q0", C.c_float), ("q1", C.c_float),
                ("encoding", C.c_int32), ("k_in", C.c_int32), ("hidden", C.c_int32),
                ("act", C.c_int32), ("out_act", C.c_int32), ("precision", C.c_int32),
                ("interp0", C.c_int32), ("lv", ntc_level * MAX_LEVELS), ("w", C.c_void_p * 3), ("b", C.c_void_p * 3),
                ("scale", C.c_void_p), ("hidden_layers", C.c_int32), ("w_h3", C.c_void_p),
                ("b_h3", C.c_void_p), ("vq_books", C.c_int32), ("codebook0", C.c_void_p)]


class ntc_grads(C.Structure):
    _fields_ = [("grid0", C.c_void_p * MAX_LEVELS), ("grid1", C.c_void_p * MAX_LEVELS),
                ("w", C.c_void_p * 3), ("b", C.c_void_p * 3), ("w_h3", C.c_void_p),
                ("b_h3", C.c_void_p)]


class ntc_trainer(C.Structure):
    _fields_ = [("params", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p),
                ("grad", C.c_void_p), ("n_params", C.c_int64), ("w_master", C.c_void_p * 3),
                ("step", C.c_void_p), ("total_steps", C.c_int64), ("lr_grid", C.c_float),
                ("lr_mlp", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("noisy", C.c_void_p), ("w_master_h3", C.c_void_p),
                ("vq_idx", C.c_void_p), ("vq_beta", C.c_float), ("noisy_tag", C.c_void_p)]


class ntc_batch(C.Structure):
    _fields_ = [("workspace", C.c_void_p), ("n_materials", C.c_int32), ("filter", C.c_int32),
                ("total_queries", C.c_int64), ("total_outputs", C.c_int64),
                ("total_tiles", C.c_int64), ("wg_smem", C.c_int32), ("fast", C.c_int32)]


class ntc_target(C.Structure):
    _fields_ = [("texels", C.c_void_p), ("offset", C.c_int64 * MAX_MIPS)]


class ntc_train_batch(C.Structure):
    _fields_ = [("workspace", C.c_void_p), ("loss_out", C.c_void_p), ("n_materials", C.c_int32),
                ("flags", C.c_int32), ("total_tiles", C.c_int64), ("adam_blocks", C.c_int64),
                ("noise_blocks", C.c_int64), ("act", C.c_int32), ("interp0", C.c_int32),
                ("hidden_layers", C.c_int32), ("k_layout", C.c_int32), ("dx_layout", C.c_int32)]


# name -> (restype, argtypes); every entry point of include/ntc.h
_P, _I32, _I64, _U64, _F = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float
SIGNATURES = {
    "ntc_version": (C.c_char_p, []),
    "ntc_last_error": (C.c_char_p, []),
    "ntc_cell_bytes": (_I32, [_I32, _I32]),
    "ntc_pyramid": (_I32, [_I32, _I32, _P, _P, _P, _P]),
    "ntc_decode": (C.c_int, [_P, _P, _I64, _P, _I32, _I32, _I32, _U64, _I64, _P]),
    "ntc_backward": (C.c_int, [_P, _P, _I64, _P, _P, _I32, _U64, _I64, _P]),
    "ntc_train_step": (C.c_int, [_P, _P, _P, _I64, _U64, _P, _P, _I32, _P]),
    "ntc_train_step_noalloc": (C.c_int, [_P, _P, _P, _I64, _U64, _P, _P, _I32, _P]),
    "ntc_quantize_pack": (C.c_int, [_P, _I64, _I32, _I32, _F, _P, _P, _P]),
    "ntc_unpack": (C.c_int, [_P, _I64, _I32, _I32, _F, _P, _P, _P]),
    "ntc_sample_batch": (C.c_int, [_U64, _I64, _I64, _I32, _I32, _I32, _P, _P]),
    "ntc_sample_crops": (C.c_int, [_U64, _I64, _I64, _I32, _I32, _I32, _P, _P]),
    "ntc_sample_features": (C.c_int, [_P, _P, _I64, _P, _I32, _U64, _I64, _P]),
    "ntc_device_status": (C.c_int, [_I32]),
    "ntc_selftest_wait": (C.c_int, [_I32, _P]),
    "ntc_batch_workspace_bytes": (C.c_size_t, []),
    "ntc_decode_host": (C.c_int, [_P, _P, _I64, _P, _I32, _I32, _I32, _U64, _I64, _P, C.c_size_t, _P]),
    "ntc_decode_host_workspace_bytes": (C.c_size_t, [_I32, _I32, _I64]),
    "ntc_vq_assign": (C.c_int, [_P, _I64, _I32, _P, _I32, _P, _P]),
    "ntc_batch_prepare": (C.c_int, [_P, _P, _I32, _I32, _P, C.c_size_t, _P, _P]),
    "ntc_decode_batched": (C.c_int, [_P, _P, _P, _I32, _P]),
    "ntc_set_decode_warpgroups": (C.c_int, [_I32]),
    "ntc_autotune_decode": (C.c_int, [_P, _P, _I64, _P, _I32, _I32, _P, _P, _P]),
    "ntc_train_batch_workspace_bytes": (C.c_size_t, []),
    "ntc_train_batch_prepare": (C.c_int, [_P, _P, _P, _P, _I32, _U64, _I32, _P, _P, C.c_size_t,
                                          _P, _P]),
    "ntc_train_step_batched": (C.c_int, [_P, _P]),
    "ntc_probe_fma_tflops": (C.c_int, [_P, _P]),
    "ntc_f8_quantize_weights": (C.c_int, [_P, _I32, _I32, _I32, _P, _P, _P]),
    "ntc_f8_activation_scales": (C.c_int, [_P, _P, _I64, _P, _P]),
    "ntc_autotune_train": (C.c_int, [_P, _P, _P, _I64, _U64, _I32, _P, _P, _P, _P]),
    "ntc_tuning_export": (C.c_int, [C.c_char_p, C.c_size_t, _P]),
    "ntc_tuning_import": (C.c_int, [C.c_char_p]),
    "ntc_tuning_clear": (C.c_int, []),
}

_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libntc.so for sm_103a (nvcc) next to this file."""
    from . import build_ext
    return build_ext.build(force=force, verbose=verbose)


def lib():
    """The loaded libntc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2305_17105_gb300.build() (there is no fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != OK:
        raise NTCError(name, rc, lib().ntc_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _queries(t: torch.Tensor, name="uvl", cuda=True) -> int:
    """Check a ``[n, 3]`` float32 contiguous query tensor; returns n."""
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3:
        raise ValueError(f"{name} must be an [n, 3] float32 tensor, got {tuple(t.shape)} {t.dtype}")
    if t.is_cuda != cuda:
        raise ValueError(f"{name} must be a {'CUDA' if cuda else 'host'} tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.shape[0]


def _room(t: torch.Tensor, name: str, elems: int, cuda=True, dtype=None):
    """Check that ``t`` (contiguous, on the right side) holds ``elems``
    elements (of ``dtype`` when given): the library writes that many."""
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < elems:
        raise ValueError(f"{name} holds {t.numel()} elements, the call uses {elems}")
    if t.is_cuda != cuda:
        raise ValueError(f"{name} must be a {'CUDA' if cuda else 'host'} tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


# ----------------------------------------------------------------------------
# small host helpers
# ----------------------------------------------------------------------------
def ntc_device_status(reset: bool = True) -> int:
    """Synchronise the device and return (and clear) the status word that
    bounded device-side waits set on timeout (OK or ERR_TIMEOUT)."""
    return int(lib().ntc_device_status(1 if reset else 0))


def ntc_selftest_wait(limit: int = 1000, stream=None) -> None:
    """Enqueue the failure-detection self-test: a bounded wait that runs out
    and records ERR_TIMEOUT in the status word (read by ntc_device_status)."""
    _call("ntc_selftest_wait", limit, _stream(stream))


def version() -> str:
    return lib().ntc_version().decode()


def cell_bytes(c: int, bits: int) -> int:
    return int(lib().ntc_cell_bytes(c, bits))


def mips_of(width: int, height: int) -> int:
    return max(width, height).bit_length()


def ntc_pyramid(width: int, height: int):
    """Feature-level grid sizes ``[((g0w, g0h), (g1w, g1h)), ...]`` (Table 1)."""
    a = [(C.c_int32 * MAX_LEVELS)() for _ in range(4)]
    n = lib().ntc_pyramid(width, height, *[C.cast(x, C.c_void_p) for x in a])
    if n == 0:
        raise ValueError("bad texture size")
    return [((a[0][j], a[1][j]), (a[2][j], a[3][j])) for j in range(n)]


pyramid = ntc_pyramid


# ----------------------------------------------------------------------------
# materials
# ----------------------------------------------------------------------------
def _layers(seq):
    """Layer-order list (3 or 4 entries) -> ([first, second, output], third
    hidden layer or None): the ABI keeps the output layer at index 2."""
    seq = list(seq)
    return ([seq[0], seq[1], seq[-1]], seq[2] if len(seq) == 4 else None)


class Material:
    """A compressed material on the device, as the C ABI sees it.

    ``grids0[j]`` / ``grids1[j]``: uint8 ``[g_h, g_w, cell_bytes]`` (packed) or
    float32 ``[g_h, g_w, c]`` (F32) CUDA tensors.  ``weights``: ``[w1, w2, w3]``
    (two hidden layers) or ``[w1, w2, w_h3, w3]`` (three), layer order,
    ``[out][in]`` tensors of the precision's dtype (float32, float16, or
    uint8 holding E4M3 bytes); ``biases`` float32, same order; ``scale`` (F8
    only) float32 ``[6]``: weight scales then activation scales.
    ``codebook0`` (vector-quantised G0) float32 ``[books, 256, c0]``: then
    ``grids0[j]`` are uint8 ``[g0_h, g0_w, books]`` indices.
    """

    def __init__(self, width, height, channels, c0, c1, bits0, bits1, q0, q1, grids0, grids1,
                 weights, biases, k_in, precision=PREC_F32, act=ACT_RELU, out_act=OUT_SIGMOID,
                 scale=None, interp0=0, codebook0=None):
        self.width, self.height, self.channels = width, height, channels
        self.mips = mips_of(width, height)
        self.c0, self.c1, self.bits0, self.bits1 = c0, c1, bits0, bits1
        self.q0, self.q1 = float(q0), float(q1)
        self.grids0, self.grids1 = list(grids0), list(grids1)
        self.weights, self.biases = list(weights), list(biases)
        assert len(self.weights) in (3, 4) and len(self.biases) == len(self.weights)
        self.k_in, self.precision, self.act, self.out_act = k_in, precision, act, out_act
        self.scale = scale
        self.interp0 = interp0
        self.codebook0 = codebook0
        self.encoding = GRID_PACKED if self.grids0[0].dtype == torch.uint8 else GRID_F32
        self.levels = len(self.grids0)

    @property
    def struct(self) -> ntc_material:
        s = ntc_material()
        s.width, s.height, s.channels, s.mips, s.levels = (self.width, self.height, self.channels,
                                                           self.mips, self.levels)
        s.c0, s.c1, s.bits0, s.bits1 = self.c0, self.c1, self.bits0, self.bits1
        s.q0, s.q1 = self.q0, self.q1
        s.encoding, s.k_in, s.hidden = self.encoding, self.k_in, HIDDEN
        s.act, s.out_act, s.precision = self.act, self.out_act, self.precision
        s.interp0 = self.interp0
        for j in range(self.levels):
            g0, g1 = self.grids0[j], self.grids1[j]
            s.lv[j].g0_h, s.lv[j].g0_w = g0.shape[0], g0.shape[1]
            s.lv[j].g1_h, s.lv[j].g1_w = g1.shape[0], g1.shape[1]
            s.lv[j].grid0, s.lv[j].grid1 = g0.data_ptr(), g1.data_ptr()
        w, b, wh, bh = _layers(self.weights), _layers(self.biases), None, None
        for l in range(3):
            s.w[l] = w[0][l].data_ptr()
            s.b[l] = b[0][l].data_ptr()
        s.hidden_layers = len(self.weights) - 1
        if w[1] is not None:
            s.w_h3, s.b_h3 = w[1].data_ptr(), b[1].data_ptr()
        s.scale = self.scale.data_ptr() if self.scale is not None else None
        if self.codebook0 is not None:
            s.vq_books, s.codebook0 = self.codebook0.shape[0], self.codebook0.data_ptr()
        return s

    def with_(self, **kw) -> "Material":
        m = Material.__new__(Material)
        m.__dict__.update(self.__dict__)
        m.__dict__.update(kw)
        if "grids0" in kw:
            m.encoding = GRID_PACKED if m.grids0[0].dtype == torch.uint8 else GRID_F32
        return m


def _out_dtype(t: torch.Tensor) -> int:
    """Output tensor dtype -> NTC_DTYPE_* (float32, float16, uint8 UNORM)."""
    if t.dtype not in _OUT_DTYPES:
        raise TypeError(f"output dtype {t.dtype}: float32, float16 or uint8")
    return _OUT_DTYPES[t.dtype]


# ----------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------
def ntc_decode(mat: Material, uvl: torch.Tensor, out_dtype=torch.float32,
               filter=FILTER_NEAREST, flags=0, noise_seed=0, noise_step=0, out=None, stream=None):
    """Decode ``uvl`` ``[n, 3]`` float32 queries -> ``[n, channels]``."""
    n = _queries(uvl)
    if out is None:
        out = torch.empty((n, mat.channels), dtype=out_dtype, device=uvl.device)
    dt = _out_dtype(out)
    _room(out, "out", n * mat.channels)
    s = mat.struct
    _call("ntc_decode", C.byref(s), _ptr(uvl), n, _ptr(out), dt, filter, flags, noise_seed,
          noise_step, _stream(stream))
    return out


def ntc_decode_host(mat: Material, uvl_host: torch.Tensor, out_host=None, out_dtype=torch.float32,
                    filter=FILTER_NEAREST, flags=0, noise_seed=0, noise_step=0, workspace=None,
                    chunk=1 << 20, stream=None):
    """Decode HOST (pinned) queries ``[n, 3]`` into a HOST output, copies and
    decode overlapped chunk by chunk through a device ``workspace`` (uint8
    CUDA tensor; allocated for ``chunk`` queries when None).  The output is
    complete once ``stream`` reaches this call's end."""
    n = _queries(uvl_host, "uvl_host", cuda=False)
    if out_host is None:
        out_host = torch.empty((n, mat.channels), dtype=out_dtype, pin_memory=True)
    dt = _out_dtype(out_host)
    _room(out_host, "out_host", n * mat.channels, cuda=False)
    if workspace is None:
        nbytes = lib().ntc_decode_host_workspace_bytes(mat.channels, dt, chunk)
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _room(workspace, "workspace", 0, dtype=torch.uint8)
    s = mat.struct
    _call("ntc_decode_host", C.byref(s), C.c_void_p(uvl_host.data_ptr()), n,
          C.c_void_p(out_host.data_ptr()), dt, filter, flags, noise_seed, noise_step,
          _ptr(workspace), workspace.numel(), _stream(stream))
    return out_host


def ntc_vq_assign(values: torch.Tensor, codebooks: torch.Tensor, stream=None) -> torch.Tensor:
    """Greedy residual vector quantisation of ``values`` ``[cells, c0]``
    against ``codebooks`` ``[books, 256, c0]`` (CUDA float32) -> uint8
    indices ``[cells, books]``."""
    if values.dim() != 2 or codebooks.dim() != 3 or codebooks.shape[1:] != (256, values.shape[1]):
        raise ValueError("values [cells, c0] and codebooks [books, 256, c0] expected")
    cells, c0 = values.shape
    books = codebooks.shape[0]
    _room(values, "values", cells * c0, dtype=torch.float32)
    _room(codebooks, "codebooks", books * 256 * c0, dtype=torch.float32)
    idx = torch.empty((cells, books), dtype=torch.uint8, device=values.device)
    _call("ntc_vq_assign", _ptr(values), cells, c0, _ptr(codebooks), books, _ptr(idx),
          _stream(stream))
    return idx


def ntc_set_decode_warpgroups(nwg: int) -> None:
    _call("ntc_set_decode_warpgroups", nwg)


def ntc_autotune_decode(mat: Material, uvl, out, filter=FILTER_NEAREST, stream=None):
    """Pick the fastest tensor-core launch shape on these queries; returns
    (best warpgroups, {shape: ms per launch})."""
    best = C.c_int32(0)
    ms = (C.c_float * 4)()
    n = _queries(uvl)
    dt = _out_dtype(out)
    _room(out, "out", n * mat.channels)
    s = mat.struct
    _call("ntc_autotune_decode", C.byref(s), _ptr(uvl), n, _ptr(out), dt, filter,
          C.byref(best), C.cast(ms, C.c_void_p), _stream(stream))
    return best.value, {2: ms[0], 3: ms[1], 4: ms[2], 5: ms[3]}


def grads_struct(mat: Material, grid0=None, grid1=None, w=None, b=None) -> ntc_grads:
    """Gradient destinations; ``w`` / ``b`` in layer order like the
    material's weights (3 or 4 entries, None entries skipped)."""
    g = ntc_grads()
    for j in range(mat.levels):
        g.grid0[j] = grid0[j].data_ptr() if grid0 is not None and grid0[j] is not None else None
        g.grid1[j] = grid1[j].data_ptr() if grid1 is not None and grid1[j] is not None else None
    ptr = lambda t: t.data_ptr() if t is not None else None
    if w is not None:
        (w3, wh) = _layers(w)
        for l in range(3):
            g.w[l] = ptr(w3[l])
        g.w_h3 = ptr(wh)
    if b is not None:
        (b3, bh) = _layers(b)
        for l in range(3):
            g.b[l] = ptr(b3[l])
        g.b_h3 = ptr(bh)
    return g


def ntc_backward(mat: Material, uvl, dout, grads: ntc_grads, flags=0, noise_seed=0, noise_step=0,
                 stream=None):
    """Accumulate d(sum dout*y)/d(grids, weights) into ``grads``."""
    n = _queries(uvl)
    _room(dout, "dout", n * mat.channels, dtype=torch.float32)
    s = mat.struct
    _call("ntc_backward", C.byref(s), _ptr(uvl), n, _ptr(dout), C.byref(grads), flags,
          noise_seed, noise_step, _stream(stream))


def ntc_quantize_pack(values: torch.Tensor, c: int, bits: int, q: float, packed=None, snapped=None,
                      want_packed=True, stream=None):
    _room(values, "values", 0, dtype=torch.float32)
    cells = values.numel() // c
    if packed is None and want_packed:
        packed = torch.empty((cells, cell_bytes(c, bits)), dtype=torch.uint8, device=values.device)
    if packed is not None:
        _room(packed, "packed", cells * cell_bytes(c, bits), dtype=torch.uint8)
    if snapped is not None:
        _room(snapped, "snapped", cells * c, dtype=torch.float32)
    _call("ntc_quantize_pack", _ptr(values), cells, c, bits, q, _ptr(packed), _ptr(snapped),
          _stream(stream))
    return packed


def ntc_unpack(packed: torch.Tensor, c: int, bits: int, q: float, want_idx=True, want_values=True,
               stream=None):
    _room(packed, "packed", 0, dtype=torch.uint8)
    cells = packed.numel() // cell_bytes(c, bits)
    idx = torch.empty((cells, c), dtype=torch.int32, device=packed.device) if want_idx else None
    val = torch.empty((cells, c), dtype=torch.float32, device=packed.device) if want_values else None
    _call("ntc_unpack", _ptr(packed), cells, c, bits, q, _ptr(idx), _ptr(val), _stream(stream))
    return idx, val


def ntc_sample_batch(seed: int, step: int, batch: int, width: int, height: int, n_mips: int,
                     device="cuda", stream=None, crops=False):
    out = torch.empty((batch, 3), dtype=torch.int32, device=device)
    _call("ntc_sample_crops" if crops else "ntc_sample_batch", seed, step, batch, width, height,
          n_mips, _ptr(out), _stream(stream))
    return out


def ntc_sample_features(mat: Material, uvl, flags=0, noise_seed=0, noise_step=0, stream=None):
    _queries(uvl)
    rows = torch.empty((uvl.shape[0], mat.k_in), dtype=torch.float32, device=uvl.device)
    s = mat.struct
    _call("ntc_sample_features", C.byref(s), _ptr(uvl), uvl.shape[0], _ptr(rows), flags,
          noise_seed, noise_step, _stream(stream))
    return rows


class Batch:
    """Materials decoded together by one persistent launch.  Keeps the
    device workspace and the prepared descriptor alive; `offsets` gives each
    material's first query row and first output element."""

    def __init__(self, materials, n_queries, filter=FILTER_NEAREST, device="cuda", stream=None):
        n = len(materials)
        self.materials = list(materials)
        arr = (ntc_material * n)()
        for i, m in enumerate(materials):
            arr[i] = m.struct
        nq = (C.c_int64 * n)(*[int(x) for x in n_queries])
        ws_bytes = lib().ntc_batch_workspace_bytes()
        self.workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        self.desc = ntc_batch()
        _call("ntc_batch_prepare", C.cast(arr, C.c_void_p), C.cast(nq, C.c_void_p), n, filter,
              _ptr(self.workspace), ws_bytes, C.byref(self.desc), _stream(stream))
        self.n_queries = [int(x) for x in n_queries]
        self.q_offsets = np.concatenate([[0], np.cumsum(self.n_queries)]).astype(np.int64)
        self.o_offsets = np.concatenate(
            [[0], np.cumsum([q * m.channels for q, m in zip(self.n_queries, materials)])]).astype(np.int64)


def ntc_decode_batched(batch: Batch, uvl, out_dtype=torch.float32, out=None, stream=None):
    _room(uvl, "uvl", 3 * int(batch.desc.total_queries), dtype=torch.float32)
    if out is None:
        out = torch.empty(int(batch.desc.total_outputs), dtype=out_dtype, device=uvl.device)
    dt = _out_dtype(out)
    _room(out, "out", int(batch.desc.total_outputs))
    _call("ntc_decode_batched", C.byref(batch.desc), _ptr(uvl), _ptr(out), dt, _stream(stream))
    return out


# ----------------------------------------------------------------------------
# training state
# ----------------------------------------------------------------------------
def _align8(n: int) -> int:
    return (n + 7) // 8 * 8


class Trainer:
    """FP32 master parameters + Adam state of one material in one flat
    device array (grids level by level, then W1, b1, W2, b2, W3, b3; every
    tensor 32-byte aligned), driven by ``ntc_train_step``."""

    def __init__(self, width, height, channels, c0, c1, bits0, bits1, q0, q1, grids0, grids1,
                 weights, biases, k_in, precision=PREC_F32, act=ACT_RELU, out_act=OUT_SIGMOID,
                 total_steps=1000, lr_grid=0.01, lr_mlp=0.005, betas=(0.9, 0.999), eps=1e-8,
                 device="cuda", noisy_scratch=True, interp0=INTERP_BILINEAR, codebook0=None,
                 vq_beta=0.25, f8_act_scales=None):
        tensors = [np.asarray(g, np.float32) for g in grids0] + \
                  [np.asarray(g, np.float32) for g in grids1]
        mlp = []
        for w, b in zip(weights, biases):
            mlp += [np.asarray(w, np.float32), np.asarray(b, np.float32)]
        tensors += mlp
        vq = codebook0 is not None
        if vq:  # vector-quantised G0: grids0 are the continuous latents, codebooks train too
            tensors.append(np.asarray(codebook0, np.float32))
        offs, n = [], 0
        for t in tensors:
            offs.append(n)
            n += _align8(t.size)
        flat = np.zeros(n, np.float32)
        for o, t in zip(offs, tensors):
            flat[o:o + t.size] = t.reshape(-1)
        self.params = torch.from_numpy(flat).to(device)
        self.adam_m = torch.zeros_like(self.params)
        self.adam_v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        # scratch for the dense noise pass of each step (None: noise per tap)
        self.noisy = torch.empty_like(self.params) if noisy_scratch else None
        # {seed, step} of the noisy copy the last step's Adam wrote
        self.noisy_tag = torch.full((2,), -1, dtype=torch.int64, device=device) \
            if noisy_scratch else None
        self.step_t = torch.zeros(1, dtype=torch.int64, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        views = [self.params[o:o + t.size].view(t.shape) for o, t in zip(offs, tensors)]
        L = len(grids0)
        self.codebook = views.pop() if vq else None
        g0, g1, rest = views[:L], views[L:2 * L], views[2 * L:]
        self.w_master = rest[0::2]   # layer order: 3 or 4 layers
        self.b = rest[1::2]
        self.grad_views = [self.grad[o:o + t.size].view(t.shape) for o, t in zip(offs, tensors)]
        self.f8_scale = None
        if precision == PREC_F16:
            self.w_compute = [w.half().contiguous() for w in self.w_master]
        elif precision == PREC_F32:
            self.w_compute = self.w_master
        elif precision == PREC_F8:
            # FP8-E4M3 form (R24): E4M3 weights the step's pre-pass writes from
            # the masters; scale = s_w[3], s_a[3], layer-input maxima[3]
            self.w_compute = [torch.zeros(w.shape, dtype=torch.uint8, device=device)
                              for w in self.w_master]
            sa = [1.0, 1.0, 1.0] if f8_act_scales is None else [float(x) for x in f8_act_scales]
            self.f8_scale = torch.tensor([1.0, 1.0, 1.0] + sa + [0.0, 0.0, 0.0],
                                         dtype=torch.float32, device=device)
        else:
            raise ValueError("precision")
        self.material = Material(width, height, channels, c0, c1, bits0, bits1, q0, q1, g0, g1,
                                 self.w_compute, self.b, k_in, precision, act, out_act,
                                 interp0=interp0, codebook0=self.codebook,
                                 scale=self.f8_scale)
        self.vq_beta = vq_beta
        self.vq_idx = (torch.empty(sum(g.shape[0] * g.shape[1] for g in grids0) * codebook0.shape[0],
                                   dtype=torch.uint8, device=device) if vq else None)
        self.total_steps, self.lr_grid, self.lr_mlp = total_steps, lr_grid, lr_mlp
        self.betas, self.eps = betas, eps

    def export(self, precision=PREC_F16, stream=None) -> Material:
        """The compressed material of the current parameters (Sec. 4.2):
        every grid value quantised to its B-bit index (bit-exact rounding)
        and packed by ``ntc_quantize_pack``; weights in the requested
        precision (FP16 or FP32) from the FP32 masters; biases copied."""
        m = self.material
        if self.codebook is not None:  # indices of the final latents, the trained codebooks
            g0 = [ntc_vq_assign(g.reshape(-1, m.c0), self.codebook, stream=stream).view(
                g.shape[0], g.shape[1], -1) for g in m.grids0]
        else:
            g0 = [ntc_quantize_pack(g.contiguous(), m.c0, m.bits0, m.q0, stream=stream).view(
                g.shape[0], g.shape[1], -1) for g in m.grids0]
        g1 = [ntc_quantize_pack(g.contiguous(), m.c1, m.bits1, m.q1, stream=stream).view(
            g.shape[0], g.shape[1], -1) for g in m.grids1]
        scale = None
        if precision == PREC_F16:
            w = [x.half().contiguous() for x in self.w_master]
        elif precision == PREC_F32:
            w = [x.clone() for x in self.w_master]
        elif precision == PREC_F8:
            # E4M3 weights with scales max|W| / 448 (ntc_f8_quantize_weights);
            # activation scales: the FP8 trainer's current ones
            if self.f8_scale is None:
                raise ValueError("FP8 export of a trainer that is not in the FP8 form")
            scale = torch.empty(6, dtype=torch.float32, device=self.params.device)
            w = [ntc_f8_quantize_weights(x.contiguous(), scale_out=scale[l:l + 1],
                                         stream=stream)[0] for l, x in enumerate(self.w_master)]
            scale[3:6] = self.f8_scale[3:6]
        else:
            raise ValueError("export writes FP8, FP16 or FP32 weights")
        return Material(m.width, m.height, m.channels, m.c0, m.c1, m.bits0, m.bits1, m.q0, m.q1,
                        g0, g1, w, [b.clone() for b in self.b], m.k_in, precision, m.act,
                        m.out_act, interp0=m.interp0,
                        codebook0=self.codebook.clone() if self.codebook is not None else None,
                        scale=scale)

    @property
    def struct(self) -> ntc_trainer:
        t = ntc_trainer()
        t.params, t.adam_m = self.params.data_ptr(), self.adam_m.data_ptr()
        t.adam_v, t.grad = self.adam_v.data_ptr(), self.grad.data_ptr()
        t.n_params = self.params.numel()
        wm, wh = _layers(self.w_master)
        for l in range(3):
            t.w_master[l] = wm[l].data_ptr()
        t.w_master_h3 = wh.data_ptr() if wh is not None else None
        t.step = self.step_t.data_ptr()
        t.total_steps = self.total_steps
        t.lr_grid, t.lr_mlp = self.lr_grid, self.lr_mlp
        t.beta1, t.beta2 = self.betas
        t.eps = self.eps
        t.noisy = self.noisy.data_ptr() if self.noisy is not None else None
        t.vq_idx = self.vq_idx.data_ptr() if self.vq_idx is not None else None
        t.vq_beta = self.vq_beta
        t.noisy_tag = self.noisy_tag.data_ptr() if self.noisy_tag is not None else None
        return t

    def invalidate_noisy(self):
        """Mark the noisy copy stale (after changing params outside the library)."""
        if self.noisy_tag is not None:
            self.noisy_tag.fill_(-1)


class Target:
    """The 8-bit reference mip chain on the device."""

    def __init__(self, mip_chain_u8, device="cuda"):
        offs, n = [], 0
        for lvl in mip_chain_u8:
            offs.append(n)
            n += (lvl.size + 15) // 16 * 16
        buf = np.zeros(n, np.uint8)
        for o, lvl in zip(offs, mip_chain_u8):
            buf[o:o + lvl.size] = np.asarray(lvl, np.uint8).reshape(-1)
        self.texels = torch.from_numpy(buf).to(device)
        self.offsets = offs

    @property
    def struct(self) -> ntc_target:
        t = ntc_target()
        t.texels = self.texels.data_ptr()
        for m, o in enumerate(self.offsets):
            t.offset[m] = o
        return t


def ntc_train_step(trainer: Trainer, target: Target, batch: int, seed: int, uvl=None, flags=0,
                   stream=None):
    """One fused optimisation step; returns the device loss tensor."""
    if uvl is not None:
        _room(uvl, "uvl", 3 * batch, dtype=torch.float32)
    m, t, tg = trainer.material.struct, trainer.struct, target.struct
    _call("ntc_train_step", C.byref(m), C.byref(t), C.byref(tg), batch, seed, _ptr(uvl),
          _ptr(trainer.loss), flags, _stream(stream))
    return trainer.loss


def ntc_train_step_noalloc(trainer: Trainer, target: Target, batch: int, seed: int, uvl=None,
                           flags=0, stream=None):
    """ntc_train_step with the scratch gradient in the library's static
    device array (no caller-provided gradient buffer; see include/ntc.h)."""
    if uvl is not None:
        _room(uvl, "uvl", 3 * batch, dtype=torch.float32)
    m, t, tg = trainer.material.struct, trainer.struct, target.struct
    t.grad = None
    _call("ntc_train_step_noalloc", C.byref(m), C.byref(t), C.byref(tg), batch, seed, _ptr(uvl),
          _ptr(trainer.loss), flags, _stream(stream))
    return trainer.loss


class TrainBatch:
    """One optimisation step of many materials per call (ntc_train_step_batched).
    ``trainers`` and ``targets`` are ``Trainer`` / ``Target`` objects (kept
    alive here), ``batches`` the texels per step of each material (0 leaves a
    material out); material i uses seed + i.  ``loss`` holds each material's
    loss after a step."""

    def __init__(self, trainers, targets, batches, seed, flags=0, device="cuda", stream=None):
        n = len(trainers)
        self.trainers, self.targets = list(trainers), list(targets)
        mats = (ntc_material * n)()
        trs = (ntc_trainer * n)()
        tgs = (ntc_target * n)()
        for i, (tr, tg) in enumerate(zip(trainers, targets)):
            mats[i], trs[i], tgs[i] = tr.material.struct, tr.struct, tg.struct
        nb = (C.c_int64 * n)(*[int(x) for x in batches])
        self.batches = [int(x) for x in batches]
        self.loss = torch.zeros(n, dtype=torch.float32, device=device)
        ws_bytes = lib().ntc_train_batch_workspace_bytes()
        self.workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        self.desc = ntc_train_batch()
        _call("ntc_train_batch_prepare", C.cast(mats, C.c_void_p), C.cast(trs, C.c_void_p),
              C.cast(tgs, C.c_void_p), C.cast(nb, C.c_void_p), n, seed, flags, _ptr(self.loss),
              _ptr(self.workspace), ws_bytes, C.byref(self.desc), _stream(stream))


def ntc_f8_quantize_weights(w, cols_out=None, scale_out=None, stream=None):
    """E4M3 bytes (uint8 [rows, cols_out]) of a float32 weight matrix and its
    scale max|w| / 448 (written into ``scale_out``, a 1-element device view,
    or a new tensor)."""
    assert w.dtype == torch.float32 and w.dim() == 2 and w.is_contiguous()
    rows, cols = w.shape
    cols_out = cols if cols_out is None else int(cols_out)
    w8 = torch.empty((rows, cols_out), dtype=torch.uint8, device=w.device)
    if scale_out is None:
        scale_out = torch.empty(1, dtype=torch.float32, device=w.device)
    _call("ntc_f8_quantize_weights", _ptr(w), rows, cols, cols_out, _ptr(w8), _ptr(scale_out),
          _stream(stream))
    return w8, scale_out


def ntc_f8_activation_scales(mat: Material, uvl, out=None, stream=None):
    """Power-of-two activation scales s_a[3] of the FP8 form from the
    per-layer input maxima of an FP32 decode of the queries ``uvl``."""
    n = _queries(uvl)
    if out is None:
        out = torch.empty(3, dtype=torch.float32, device=uvl.device)
    s = mat.struct
    _call("ntc_f8_activation_scales", C.byref(s), _ptr(uvl), n, _ptr(out), _stream(stream))
    return out


def f8_material(mat: Material, w32, calib_uvl, stream=None) -> Material:
    """The FP8-E4M3 form of a material: E4M3 weights with per-layer scales
    (ntc_f8_quantize_weights on the FP32 weights ``w32``, layer order) and
    activation scales calibrated on the queries ``calib_uvl``
    (ntc_f8_activation_scales); K rounded up to a multiple of 32."""
    k8 = (mat.k_in + 31) // 32 * 32
    dev = calib_uvl.device
    scale = torch.empty(6, dtype=torch.float32, device=dev)
    w8 = []
    for l, w in enumerate(w32):
        wt = torch.as_tensor(w, dtype=torch.float32, device=dev).contiguous()
        q, _ = ntc_f8_quantize_weights(wt, k8 if l == 0 else wt.shape[1], scale[l:l + 1],
                                       stream=stream)
        w8.append(q)
    ntc_f8_activation_scales(mat, calib_uvl, out=scale[3:6], stream=stream)
    return mat.with_(weights=w8, precision=PREC_F8, scale=scale, k_in=k8)


def ntc_autotune_train(trainer: Trainer, target: Target, batch: int, seed: int, flags=0,
                       stream=None):
    """Time the fused step with 1-3 pipelines per CTA and record the fastest
    in the tuning cache; returns (best, [ms for 1, 2, 3])."""
    m, t, tg = trainer.material.struct, trainer.struct, target.struct
    best = C.c_int32(0)
    ms = (C.c_float * 3)()
    _call("ntc_autotune_train", C.byref(m), C.byref(t), C.byref(tg), batch, seed, flags,
          _ptr(trainer.loss), C.byref(best), ms, _stream(stream))
    return int(best.value), [float(x) for x in ms]


def tuning_export() -> str:
    """The tuning cache as text (one "<key> <value>" line per entry)."""
    n = C.c_size_t(0)
    _call("ntc_tuning_export", None, 0, C.byref(n))
    buf = C.create_string_buffer(int(n.value))
    _call("ntc_tuning_export", buf, int(n.value), C.byref(n))
    return buf.value.decode()


def tuning_import(text: str) -> None:
    _call("ntc_tuning_import", text.encode())


def tuning_clear() -> None:
    _call("ntc_tuning_clear")


def tuning_save(path: str) -> None:
    with open(path, "w") as f:
        f.write(tuning_export())


def tuning_load(path: str) -> None:
    with open(path) as f:
        tuning_import(f.read())


def ntc_probe_fma_tflops(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s)."""
    v = C.c_float(0.0)
    _call("ntc_probe_fma_tflops", C.byref(v), _stream(stream))
    return float(v.value)


def ntc_train_step_batched(batch: TrainBatch, stream=None):
    """One step of every material of the batch; returns the device loss
    tensor [n_materials]."""
    _call("ntc_train_step_batched", C.byref(batch.desc), _stream(stream))
    return batch.loss


# ----------------------------------------------------------------------------
# autograd
# ----------------------------------------------------------------------------
class NTCDecodeFunction(torch.autograd.Function):
    """Nearest decode with a hand-written adjoint: ``ntc_decode`` forward,
    ``ntc_backward`` backward (recomputes activations; scatter-adds into the
    latent grids; the simulated-quantisation noise passes gradients).  FP16
    materials run the tensor-core adjoint, FP32 ones the CUDA-core adjoint.
    Weights and biases come in layer order, 3 layers (two hidden) or 4
    (three hidden)."""

    @staticmethod
    def forward(ctx, uvl, mat_proto, noise, n_layers, *tensors):
        L = mat_proto.levels
        g0, g1 = list(tensors[:L]), list(tensors[L:2 * L])
        w = list(tensors[2 * L:2 * L + n_layers])
        b = list(tensors[2 * L + n_layers:2 * L + 2 * n_layers])
        wc = [x.half().contiguous() for x in w] if mat_proto.precision == PREC_F16 else w
        mat = mat_proto.with_(grids0=g0, grids1=g1, weights=wc, biases=b)
        flags = FLAG_NOISE if noise is not None else 0
        seed, step = noise if noise is not None else (0, 0)
        y = ntc_decode(mat, uvl, flags=flags, noise_seed=seed, noise_step=step)
        ctx.save_for_backward(uvl, *tensors)
        ctx.mat, ctx.flags, ctx.seed, ctx.step, ctx.L, ctx.nl = mat, flags, seed, step, L, n_layers
        return y

    @staticmethod
    def backward(ctx, dy):
        uvl, *tensors = ctx.saved_tensors
        L, nl = ctx.L, ctx.nl
        grads = [torch.zeros_like(t) for t in tensors]
        gs = grads_struct(ctx.mat, grads[:L], grads[L:2 * L], grads[2 * L:2 * L + nl],
                          grads[2 * L + nl:2 * L + 2 * nl])
        ntc_backward(ctx.mat, uvl, dy.contiguous().float(), gs, flags=ctx.flags,
                     noise_seed=ctx.seed, noise_step=ctx.step)
        return (None, None, None, None, *grads)


def decode_autograd(mat_proto: Material, uvl, grids0, grids1, weights, biases, noise=None):
    assert len(weights) == len(biases) and len(weights) in (3, 4)
    return NTCDecodeFunction.apply(uvl, mat_proto, noise, len(weights), *grids0, *grids1,
                                   *weights, *biases)
