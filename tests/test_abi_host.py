"""Host-side checks of the C ABI: the library builds and loads, exports every
entry point that include/ntc.h declares, and its host logic (pyramid rule,
cell sizes, argument validation) behaves -- no GPU needed: every call here
returns before any CUDA work is enqueued."""
import ctypes as C
import os
import re

import pytest
import torch

import oracle
import paper_2305_17105_gb300 as ntc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ntc.LIB_PATH):
        ntc.build()
    return ntc.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "ntc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ntc_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert "ntc_decode" in names and "ntc_train_step" in names and "ntc_backward" in names
    for n in names:
        assert hasattr(L, n), n
    # and the binding wraps each of them
    assert set(names) <= set(ntc.SIGNATURES)


def test_version(L):
    assert "sm_103a" in ntc.version()


@pytest.mark.parametrize("c,bits", [(8, 4), (12, 4), (16, 4), (8, 2), (12, 2), (20, 4), (3, 4),
                                    (5, 8), (7, 1), (16, 8)])
def test_cell_bytes_matches_oracle(L, c, bits):
    assert ntc.cell_bytes(c, bits) == oracle.cell_bytes(c, bits)


def test_cell_bytes_rejects(L):
    assert ntc.cell_bytes(0, 4) == 0 and ntc.cell_bytes(8, 3) == 0 and ntc.cell_bytes(17, 8) == 0


@pytest.mark.parametrize("w,h", [(1, 1), (2, 2), (8, 8), (16, 16), (64, 32), (256, 256),
                                 (1024, 1024), (2048, 2048), (4096, 4096), (8192, 8192),
                                 (512, 4096), (32768, 32768)])
def test_pyramid_matches_oracle(L, w, h):
    assert ntc.pyramid(w, h) == oracle.pyramid(w, h)


def _fake_material(**kw):
    """A well-formed material struct whose device pointers are fake but
    aligned: only argument validation may look at it."""
    m = ntc.ntc_material()
    m.width = m.height = 64
    m.channels, m.mips, m.levels = 4, 7, 2
    m.c0 = m.c1 = 8
    m.bits0 = m.bits1 = 4
    m.q0 = m.q1 = 1 / 16
    m.encoding, m.k_in, m.hidden = ntc.GRID_PACKED, 32, 64
    m.act, m.out_act, m.precision = 0, 0, ntc.PREC_F32
    for j in range(2):
        m.lv[j].g0_w = m.lv[j].g0_h = 16 >> (2 * j)
        m.lv[j].g1_w = m.lv[j].g1_h = 8 >> (2 * j)
        m.lv[j].grid0 = m.lv[j].grid1 = 0x10000
    for l in range(3):
        m.w[l] = m.b[l] = 0x20000
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def _decode_rc(L, m, n=0, uvl=0x30000, out=0x40000, out_dtype=0, filt=0, flags=0):
    return L.ntc_decode(C.byref(m) if m is not None else None, uvl, n, out, out_dtype, filt, flags,
                        0, 0, None)


def test_valid_material_with_zero_queries_is_a_noop(L):
    assert _decode_rc(L, _fake_material(), n=0) == ntc.OK


@pytest.mark.parametrize("kw,code", [
    (dict(width=63), ntc.ERR_SHAPE),
    (dict(mips=6), ntc.ERR_SHAPE),
    (dict(channels=17), ntc.ERR_SHAPE),
    (dict(channels=0), ntc.ERR_SHAPE),
    (dict(levels=0), ntc.ERR_SHAPE),
    (dict(levels=9), ntc.ERR_SHAPE),
    (dict(c0=17), ntc.ERR_SHAPE),
    (dict(bits0=3), ntc.ERR_ARG),
    (dict(q1=0.0), ntc.ERR_ARG),
    (dict(k_in=24), ntc.ERR_SHAPE),       # not a multiple of 16
    (dict(k_in=16), ntc.ERR_SHAPE),       # < c0 + c1 + 13
    (dict(k_in=144), ntc.ERR_SHAPE),
    (dict(hidden=32), ntc.ERR_UNSUPPORTED),
    (dict(act=5), ntc.ERR_ARG),
    (dict(out_act=3), ntc.ERR_ARG),
    (dict(precision=7), ntc.ERR_ARG),
    (dict(encoding=4), ntc.ERR_ARG),
    (dict(hidden_layers=4), ntc.ERR_ARG),
    (dict(hidden_layers=1), ntc.ERR_ARG),
    (dict(hidden_layers=3), ntc.ERR_ARG),                  # w_h3 / b_h3 missing
    (dict(hidden_layers=3, w_h3=0x20000, b_h3=0x20000, precision=ntc.PREC_F8, k_in=64,
          scale=0x20000), ntc.ERR_UNSUPPORTED),
    (dict(vq_books=5, codebook0=0x20000), ntc.ERR_ARG),
    (dict(vq_books=2), ntc.ERR_ARG),                       # codebook missing
    (dict(vq_books=2, codebook0=0x20000, precision=ntc.PREC_F8, k_in=64, scale=0x20000),
     ntc.ERR_UNSUPPORTED),
])
def test_material_validation(L, kw, code):
    assert _decode_rc(L, _fake_material(**kw), n=5) == code
    assert L.ntc_last_error().decode()


def test_three_hidden_layers_valid_material_is_a_noop(L):
    m = _fake_material(hidden_layers=3, w_h3=0x20000, b_h3=0x20000)
    assert _decode_rc(L, m, n=0) == ntc.OK


def test_decode_host_validation(L):
    L.ntc_decode_host.restype = C.c_int
    L.ntc_decode_host.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                  C.c_int32, C.c_int32, C.c_uint64, C.c_int64, C.c_void_p,
                                  C.c_size_t, C.c_void_p]
    L.ntc_decode_host_workspace_bytes.restype = C.c_size_t
    L.ntc_decode_host_workspace_bytes.argtypes = [C.c_int32, C.c_int32, C.c_int64]
    m = C.byref(_fake_material())
    host = (C.c_float * 30)()
    ok = L.ntc_decode_host_workspace_bytes(4, ntc.DTYPE_F16, 128)
    assert ok == 2 * 128 * (12 + 4 * 2)
    assert L.ntc_decode_host_workspace_bytes(0, 0, 128) == 0
    assert L.ntc_decode_host_workspace_bytes(4, ntc.DTYPE_U8, 128) == 2 * 128 * (12 + 4)
    assert L.ntc_decode_host_workspace_bytes(4, 3, 128) == 0
    args = lambda **kw: dict(dict(uvl=C.addressof(host), n=10, out=C.addressof(host), dt=0, f=0,
                                  ws=0x50000, wsb=ok * 2), **kw)
    def rc(a):
        return L.ntc_decode_host(m, a["uvl"], a["n"], a["out"], a["dt"], a["f"], 0, 0, 0, a["ws"],
                                 a["wsb"], None)
    assert rc(args(n=0)) == ntc.OK
    assert rc(args(f=ntc.FILTER_STOCHASTIC)) == ntc.ERR_UNSUPPORTED
    assert rc(args(uvl=None)) == ntc.ERR_ARG
    assert rc(args(ws=None)) == ntc.ERR_ARG
    assert rc(args(ws=0x50004)) == ntc.ERR_ALIGN
    assert rc(args(wsb=ok // 2)) == ntc.ERR_ARG     # below two 128-query chunks
    assert rc(args(dt=7)) == ntc.ERR_ARG


def test_selftest_wait_validation(L):
    assert L.ntc_selftest_wait(0, None) == ntc.ERR_ARG
    assert L.ntc_selftest_wait((1 << 20) + 1, None) == ntc.ERR_ARG


def test_pointer_validation(L):
    assert _decode_rc(L, None, n=5) == ntc.ERR_ARG
    assert _decode_rc(L, _fake_material(), n=5, uvl=0x30004) == ntc.ERR_ALIGN
    assert _decode_rc(L, _fake_material(), n=5, out=0) == ntc.ERR_ARG
    m = _fake_material()
    m.lv[1].grid1 = 0x10008
    assert _decode_rc(L, m, n=5) == ntc.ERR_ALIGN
    assert _decode_rc(L, _fake_material(), n=-1) == ntc.ERR_ARG
    assert _decode_rc(L, _fake_material(), n=5, out_dtype=9) == ntc.ERR_ARG
    assert _decode_rc(L, _fake_material(), n=5, out_dtype=3) == ntc.ERR_ARG
    assert _decode_rc(L, _fake_material(), n=5, filt=9) == ntc.ERR_ARG
    # noise needs F32 grids
    assert _decode_rc(L, _fake_material(), n=5, flags=ntc.FLAG_NOISE) == ntc.ERR_ARG
    # FP8 needs 32-aligned K and a scale pointer
    assert _decode_rc(L, _fake_material(precision=ntc.PREC_F8, k_in=48), n=5) == ntc.ERR_SHAPE
    assert _decode_rc(L, _fake_material(precision=ntc.PREC_F8, k_in=64), n=5) == ntc.ERR_ARG


def test_train_step_validation(L):
    m = _fake_material(encoding=ntc.GRID_F32)
    tr = ntc.ntc_trainer()
    tg = ntc.ntc_target()
    loss = C.c_void_p(0x50000)
    # packed grids are not trainable
    rc = L.ntc_train_step(C.byref(_fake_material()), C.byref(tr), C.byref(tg), 16, 1, None, loss, 0, None)
    assert rc == ntc.ERR_ARG
    # missing trainer buffers
    rc = L.ntc_train_step(C.byref(m), C.byref(tr), C.byref(tg), 16, 1, None, loss, 0, None)
    assert rc == ntc.ERR_ARG
    tr.params = tr.adam_m = tr.adam_v = tr.grad = 0x100000
    tr.step = 0x200000
    tg.texels = 0x300000
    tr.total_steps = 10
    for l in range(3):
        tr.w_master[l] = 0x20000
    tr.n_params = 16
    # grids do not lie inside params
    rc = L.ntc_train_step(C.byref(m), C.byref(tr), C.byref(tg), 16, 1, None, loss, 0, None)
    assert rc == ntc.ERR_ARG and "params" in L.ntc_last_error().decode()
    rc = L.ntc_train_step(C.byref(m), C.byref(tr), C.byref(tg), 0, 1, None, loss, 0, None)
    assert rc == ntc.ERR_ARG
    # the FP8 form trains on the tensor cores only, bilinear G0, K in 32s
    m8 = _fake_material(encoding=ntc.GRID_F32, precision=ntc.PREC_F8, scale=0x20000)
    rc = L.ntc_train_step(C.byref(m8), C.byref(tr), C.byref(tg), 16, 1, None, loss,
                          ntc.FLAG_SIMT, None)
    assert rc == ntc.ERR_UNSUPPORTED
    m8l = _fake_material(encoding=ntc.GRID_F32, precision=ntc.PREC_F8, scale=0x20000, k_in=64,
                         act=ntc.ACT_HARDGELU)
    rc = L.ntc_train_step(C.byref(m8l), C.byref(tr), C.byref(tg), 16, 1, None, loss, 0, None)
    assert rc == ntc.ERR_ARG and "params" in L.ntc_last_error().decode()  # passes the FP8 checks


def test_tuning_cache_text(L):
    """The tuning cache's text form: import, export and clear are host-only;
    malformed lines and values outside 1..5 are refused."""
    ntc.tuning_clear()
    ntc.tuning_import("train:k=1 2\ndecode:k=2 5\n\n")
    text = ntc.tuning_export()
    assert text == "decode:k=2 5\ntrain:k=1 2\n"
    for bad in ("novalue\n", "train:k=1 9\n", "train:k=1 x\n"):
        with pytest.raises(ntc.NTCError):
            ntc.tuning_import(bad)
    assert ntc.tuning_export() == text  # a refused import adds nothing
    ntc.tuning_clear()
    assert ntc.tuning_export() == ""


def test_grid_width_rules(L):
    """Grids hold 1..20 features per cell (profile 0.5's G1 has 20), packed
    cells at most 128 bits."""
    assert _decode_rc(L, _fake_material(c0=12, c1=20, k_in=48), n=0) == ntc.OK
    assert _decode_rc(L, _fake_material(c0=21, c1=8, k_in=48), n=0) == ntc.ERR_SHAPE
    assert _decode_rc(L, _fake_material(c0=20, c1=8, bits0=8, k_in=48), n=0) == ntc.ERR_SHAPE
    assert _decode_rc(L, _fake_material(c0=16, c1=8, bits0=8, k_in=48), n=0) == ntc.OK
    f32 = _fake_material(c0=20, c1=8, bits0=8, k_in=48, encoding=ntc.GRID_F32)
    assert _decode_rc(L, f32, n=0) == ntc.OK


def test_noalloc_step_refuses_gradient_only(L):
    """The allocation-free step keeps its gradient in a private array, so a
    gradient-only call (whose only result is that gradient) is refused
    before any CUDA call."""
    m = _fake_material(encoding=ntc.GRID_F32)
    tr = ntc.ntc_trainer()
    tr.n_params = 16
    rc = L.ntc_train_step_noalloc(C.byref(m), C.byref(tr), C.byref(ntc.ntc_target()), 16, 1, None,
                                  C.c_void_p(0x50000), ntc.FLAG_GRAD_ONLY, None)
    assert rc == ntc.ERR_ARG and "GRAD_ONLY" in L.ntc_last_error().decode()
    assert L.ntc_train_step_noalloc(C.byref(m), None, None, 16, 1, None, None, 0, None) == ntc.ERR_ARG


def test_train_batch_validation(L):
    """ntc_train_batch_prepare refuses, before any CUDA call: an empty or
    oversized batch, flags outside FREEZE_GRIDS / NO_NOISE / CROPS /
    GRAD_ONLY, FP32 materials, materials of different kernel classes, a
    trainer used twice, negative batches and a short workspace."""
    n = 2
    mats = (ntc.ntc_material * n)(*[_fake_material(encoding=ntc.GRID_F32, precision=ntc.PREC_F16)
                                    for _ in range(n)])
    trs = (ntc.ntc_trainer * n)()
    tgs = (ntc.ntc_target * n)()
    for i in range(n):
        trs[i].params = 0x100000 * (i + 1)
        trs[i].step = 0x900000 + 0x100 * i
    nb = (C.c_int64 * n)(100, 0)
    ws_bytes = L.ntc_train_batch_workspace_bytes()
    assert ws_bytes > 0
    out = ntc.ntc_train_batch()

    def rc(mats_=mats, trs_=trs, nb_=nb, count=n, flags=0, ws=0x700000, wsb=ws_bytes):
        return L.ntc_train_batch_prepare(C.cast(mats_, C.c_void_p), C.cast(trs_, C.c_void_p),
                                         C.cast(tgs, C.c_void_p), C.cast(nb_, C.c_void_p), count,
                                         1, flags, C.c_void_p(0x800000), ws, wsb, C.byref(out),
                                         None)

    assert rc(count=0) == ntc.ERR_ARG
    assert rc(count=ntc.MAX_TRAIN_BATCH + 1) == ntc.ERR_ARG
    assert rc(flags=ntc.FLAG_SIMT) == ntc.ERR_ARG
    assert rc(wsb=ws_bytes - 1) == ntc.ERR_ARG
    mats[1].precision = ntc.PREC_F32
    assert rc() == ntc.ERR_UNSUPPORTED and "FP16" in L.ntc_last_error().decode()
    mats[1].precision = ntc.PREC_F16
    mats[1].act = ntc.ACT_HARDGELU
    assert rc() == ntc.ERR_UNSUPPORTED and "shares" in L.ntc_last_error().decode()
    mats[1].act = ntc.ACT_RELU
    nb[1] = -1
    assert rc() == ntc.ERR_ARG
    nb[1] = 0
    trs[1].params = trs[0].params
    assert rc() == ntc.ERR_ARG and "share a trainer" in L.ntc_last_error().decode()
    trs[1].params = 0x200000
    # the per-material checks of ntc_train_step apply (no Adam state here)
    assert rc() == ntc.ERR_ARG and "material 0" in L.ntc_last_error().decode()
    assert L.ntc_train_step_batched(None, None) == ntc.ERR_ARG


def test_quantize_and_sampler_validation(L):
    assert L.ntc_quantize_pack(0x1000, 10, 8, 3, 0.0625, 0x2000, None, None) == ntc.ERR_ARG
    assert L.ntc_quantize_pack(0x1000, 10, 8, 4, 0.0, 0x2000, None, None) == ntc.ERR_ARG
    assert L.ntc_quantize_pack(0x1004, 10, 8, 4, 0.0625, 0x2000, None, None) == ntc.ERR_ALIGN
    assert L.ntc_quantize_pack(0x1000, 0, 8, 4, 0.0625, 0x2000, None, None) == ntc.OK
    assert L.ntc_unpack(0x1000, 10, 8, 4, 0.0625, 0x2004, None, None) == ntc.ERR_ALIGN
    assert L.ntc_sample_batch(1, 0, 10, 48, 64, 7, 0x1000, None) == ntc.ERR_ARG
    assert L.ntc_sample_batch(1, 0, 10, 64, 64, 17, 0x1000, None) == ntc.ERR_ARG
    assert L.ntc_sample_batch(1, 0, 0, 64, 64, 7, 0x1000, None) == ntc.OK
    assert L.ntc_sample_crops(1, 0, 10, 48, 64, 7, 0x1000, None) == ntc.ERR_ARG
    assert L.ntc_sample_crops(1, 0, 0, 64, 64, 7, 0x1000, None) == ntc.OK


def test_autotune_validation(L):
    L.ntc_autotune_decode.restype = C.c_int
    L.ntc_autotune_decode.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                      C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    best = C.c_int32(0)
    m = C.byref(_fake_material())
    rc = lambda dt=0, f=0, n=5: L.ntc_autotune_decode(m, 0x30000, n, 0x40000, dt, f,
                                                       C.byref(best), None, None)
    assert rc(dt=3) == ntc.ERR_ARG
    assert rc(f=9) == ntc.ERR_ARG
    assert rc(n=0) == ntc.ERR_ARG


def test_binding_rejects_unknown_output_dtype():
    for dt in (torch.float64, torch.int32, torch.bfloat16):
        with pytest.raises(TypeError):
            ntc._out_dtype(torch.empty(1, dtype=dt))
    assert ntc._out_dtype(torch.empty(1, dtype=torch.uint8)) == ntc.DTYPE_U8


def test_binding_checks_shapes_before_any_launch():
    """The binding refuses tensors the library would read or write past
    their end, before it calls into the library (the host-side cases; the
    device-buffer cases are GPU tests)."""
    class M:
        channels = 4
        k_in = 32
    with pytest.raises(ValueError, match=r"\[n, 3\] float32"):
        ntc.ntc_decode(M, torch.zeros(10, 2))
    with pytest.raises(ValueError, match=r"\[n, 3\] float32"):
        ntc.ntc_decode(M, torch.zeros(10, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="uvl must be a CUDA tensor"):
        ntc.ntc_decode(M, torch.zeros(10, 3))
    with pytest.raises(ValueError, match="uvl must be a CUDA tensor"):
        ntc.ntc_backward(M, torch.zeros(10, 3), torch.zeros(40), None)
    with pytest.raises(ValueError, match="the call uses 40"):
        ntc.ntc_decode_host(M, torch.zeros(10, 3), out_host=torch.zeros(39))
    with pytest.raises(TypeError):
        ntc.ntc_decode_host(M, torch.zeros(10, 3), out_host=torch.zeros(40, dtype=torch.int16))
    with pytest.raises(ValueError, match="codebooks"):
        ntc.ntc_vq_assign(torch.zeros(5, 8), torch.zeros(2, 255, 8))


def test_backward_validation(L):
    g = ntc.ntc_grads()
    m32 = _fake_material(encoding=ntc.GRID_F32)

    def rc(m, n=5, uvl=0x30000, dout=0x40000, grads=True):
        return L.ntc_backward(C.byref(m), uvl, n, dout, C.byref(g) if grads else None, 0, 0, 0,
                              None)
    assert rc(_fake_material()) == ntc.ERR_ARG          # packed grids are not differentiable
    assert rc(m32, n=-1) == ntc.ERR_ARG
    assert rc(m32, grads=False) == ntc.ERR_ARG
    assert rc(m32, n=0) == ntc.OK
    assert rc(m32, uvl=0x30004) == ntc.ERR_ALIGN
    assert rc(m32, dout=None) == ntc.ERR_ARG
    g.grid0[1] = 0x60008
    assert rc(m32) == ntc.ERR_ALIGN
    g.grid0[1] = None
    assert rc(_fake_material(encoding=ntc.GRID_F32, hidden_layers=3, w_h3=0x20000,
                             b_h3=0x20000)) == ntc.ERR_UNSUPPORTED


def test_batch_validation(L):
    arr = (ntc.ntc_material * 2)(_fake_material(precision=ntc.PREC_F16),
                                 _fake_material(precision=ntc.PREC_F16))
    nq = (C.c_int64 * 2)(10, 20)
    desc = ntc.ntc_batch()
    ws_bytes = L.ntc_batch_workspace_bytes()

    def rc(a=arr, q=nq, n=2, f=ntc.FILTER_NEAREST, ws=0x100000, wsb=ws_bytes, d=True):
        return L.ntc_batch_prepare(C.cast(a, C.c_void_p) if a is not None else None,
                                   C.cast(q, C.c_void_p) if q is not None else None, n, f, ws, wsb,
                                   C.byref(desc) if d else None, None)
    assert rc(a=None) == ntc.ERR_ARG and rc(q=None) == ntc.ERR_ARG and rc(d=False) == ntc.ERR_ARG
    assert rc(n=0) == ntc.ERR_ARG
    assert rc(f=ntc.FILTER_STOCHASTIC) == ntc.ERR_ARG
    assert rc(ws=0x100008) == ntc.ERR_ALIGN
    assert rc(wsb=ws_bytes - 1) == ntc.ERR_ARG
    nq[1] = -1
    assert rc() == ntc.ERR_ARG
    nq[1] = 1 << 31                                     # a material's queries must fit 31 bits
    assert rc() == ntc.ERR_SHAPE
    nq[1] = 20
    # and a batch's tiles: 200 materials of 2^31 - 1 queries
    many = (ntc.ntc_material * 200)(*[_fake_material(precision=ntc.PREC_F16)] * 200)
    big = (C.c_int64 * 200)(*[(1 << 31) - 1] * 200)
    assert rc(a=many, q=big, n=200) == ntc.ERR_SHAPE
    assert "tiles" in L.ntc_last_error().decode()
    arr[1] = _fake_material()                           # FP32 weights: not batched
    assert rc() == ntc.ERR_UNSUPPORTED
    # decode of an unprepared or empty batch
    assert L.ntc_decode_batched(C.byref(ntc.ntc_batch()), 0x30000, 0x40000, 0, None) == ntc.ERR_ARG
    empty = ntc.ntc_batch()
    empty.workspace = 0x100000
    assert L.ntc_decode_batched(C.byref(empty), 0x30000, 0x40000, 3, None) == ntc.ERR_ARG
    assert L.ntc_decode_batched(C.byref(empty), 0x30000, 0x40000, ntc.DTYPE_U8, None) == ntc.OK


def test_vq_features_and_shape_validation(L):
    assert L.ntc_vq_assign(0x1000, -1, 8, 0x2000, 2, 0x3000, None) == ntc.ERR_ARG
    assert L.ntc_vq_assign(0x1000, 10, 0, 0x2000, 2, 0x3000, None) == ntc.ERR_ARG
    assert L.ntc_vq_assign(0x1000, 10, 8, 0x2000, 5, 0x3000, None) == ntc.ERR_ARG
    assert L.ntc_vq_assign(0x1000, 0, 8, 0x2000, 2, 0x3000, None) == ntc.OK
    assert L.ntc_vq_assign(0x1004, 10, 8, 0x2000, 2, 0x3000, None) == ntc.ERR_ALIGN
    assert L.ntc_vq_assign(0x1000, 10, 8, 0x2000, 2, None, None) == ntc.ERR_ARG
    m = C.byref(_fake_material())
    assert L.ntc_sample_features(m, 0x1000, -1, 0x2000, 0, 0, 0, None) == ntc.ERR_ARG
    assert L.ntc_sample_features(m, 0x1000, 0, 0x2000, 0, 0, 0, None) == ntc.OK
    assert L.ntc_sample_features(m, 0x1000, 5, 0x2004, 0, 0, 0, None) == ntc.ERR_ALIGN
    assert L.ntc_sample_features(m, 0x1000, 5, 0x2000, ntc.FLAG_NOISE, 0, 0, None) == ntc.ERR_ARG
    assert L.ntc_set_decode_warpgroups(1) == ntc.ERR_ARG
    assert L.ntc_set_decode_warpgroups(6) == ntc.ERR_ARG
    assert L.ntc_set_decode_warpgroups(5) == ntc.OK and L.ntc_set_decode_warpgroups(0) == ntc.OK


def _header_constants():
    """NTC_* values from include/ntc.h: enum members (explicit values) and
    integer #defines (shifts evaluated)."""
    src = open(os.path.join(ROOT, "include", "ntc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(NTC_[A-Z0-9_]+)\s*=\s*([^,}\n]+)", body):
            out[name] = int(eval(val.strip(), {}, {}))
    for name, val in re.findall(r"#define\s+(NTC_[A-Z0-9_]+)\s+\(?([0-9x<> ]+)\)?", src):
        out[name] = int(eval(val.strip(), {}, {}))
    return out


def test_binding_constants_match_the_header():
    consts = _header_constants()
    assert len(consts) > 30
    alias = {"NTC_MAX_LEVELS": "MAX_LEVELS", "NTC_MAX_MIPS": "MAX_MIPS",
             "NTC_MAX_CHANNELS": "MAX_CHANNELS", "NTC_MAX_K": "MAX_K", "NTC_HIDDEN": "HIDDEN"}
    checked = 0
    for name, val in consts.items():
        py = alias.get(name, name[len("NTC_"):])
        if hasattr(ntc, py):
            assert getattr(ntc, py) == val, (name, getattr(ntc, py), val)
            checked += 1
    for must in ("NTC_DTYPE_U8", "NTC_FLAG_CROPS", "NTC_FILTER_STOCHASTIC", "NTC_PREC_F8",
                 "NTC_ERR_TIMEOUT", "NTC_INTERP_LEARNED", "NTC_GRID_F32"):
        assert must in consts and hasattr(ntc, must[len("NTC_"):]), must
    assert checked == len(consts)


def test_struct_layouts_match_the_header():
    """sizeof and every field offset of the ABI structs, compiled from
    include/ntc.h by the host C compiler, equal the binding's ctypes
    layouts (a drifted field would silently shift every later one)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [ntc.ntc_level, ntc.ntc_material, ntc.ntc_grads, ntc.ntc_trainer, ntc.ntc_target,
               ntc.ntc_batch]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ntc.h"', "int main(void) {"]
    for st in structs:
        nm = st.__name__
        lines.append(f'  printf("{nm} sizeof %zu\\n", sizeof({nm}));')
        for f in st._fields_:
            lines.append(f'  printf("{nm} {f[0]} %zu\\n", offsetof({nm}, {f[0]}));')
    lines += ["  return 0;", "}"]
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "abi_layout.c"), os.path.join(out_dir, "abi_layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True)
    got = {}
    for line in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for st in structs:
        nm = st.__name__
        assert got[(nm, "sizeof")] == C.sizeof(st), nm
        for f in st._fields_:
            assert got[(nm, f[0])] == getattr(st, f[0]).offset, (nm, f[0])


def _prototypes():
    """name -> (return type, [parameter types]) of every function in
    include/ntc.h (comments stripped, parameter names dropped)."""
    src = open(os.path.join(ROOT, "include", "ntc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(ntc_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;",
                                        src, flags=re.S):
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        types = [re.sub(r"\s*\b\w+\s*$", "", p) if not p.endswith("*") else p for p in ps]
        out[name] = (ret.strip().split()[-1] if ret.strip() else ret, types)
    return out


def _ctype_of(ctype: str):
    t = " ".join(ctype.replace("const ", "").split())
    if "*" in t:
        return C.c_char_p if t == "char*" or t == "char *" else C.c_void_p
    return {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "float": C.c_float,
            "size_t": C.c_size_t, "int": C.c_int}[t]


def test_binding_signatures_match_the_prototypes():
    """Every entry point's ctypes argtypes are the header's parameter types
    in order (a 32-bit argtype for a 64-bit parameter would pass garbage)."""
    protos = _prototypes()
    assert set(protos) == set(ntc.SIGNATURES), set(protos) ^ set(ntc.SIGNATURES)
    for name, (ret, types) in protos.items():
        rw, rg = _ctype_of(ret), ntc.SIGNATURES[name][0]
        assert C.sizeof(rg) == C.sizeof(rw) and (rw is C.c_char_p) == (rg is C.c_char_p), name
        want = [_ctype_of(t) for t in types]
        got = ntc.SIGNATURES[name][1]
        assert len(got) == len(want), (name, len(got), len(want))
        for i, (g, w) in enumerate(zip(got, want)):
            assert C.sizeof(g) == C.sizeof(w) and (g in (C.c_float,)) == (w in (C.c_float,)), \
                (name, i, g, w)
            if w is C.c_void_p:
                assert g is C.c_void_p, (name, i)
