"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *generates data*: textures, latent-grid initial values, MLP
initial weights, decode queries and camera queries.  It holds none of the
neural-texture-compression arithmetic (no feature-level selection, no
quantisation, no interpolation, no MLP): both the CPU oracle and the CUDA
library receive these arrays as plain inputs and compute on them
independently.

The paper evaluates on a 20-material dataset of 2k-8k texture sets with 3-12
channels (Sec. 6.1, App. I) that is not available here.  The generators below
stand in for it with the same shapes and channel counts: smooth multi-octave
value noise mixed across channels so that channels are strongly correlated
(the low-rank cross-channel structure that Sec. 3 motivates the method with).

Seed convention: material ``1000 + id``, MLP init ``2000 + id``, training
sampler ``3000 + id``, decode queries ``4000 + id``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "value_noise",
    "synthetic_texture",
    "box_mip_chain_u8",
    "uniform_grid_values",
    "random_mlp",
    "random_queries",
    "random_texel_queries",
    "camera_queries",
    "material_set_shapes",
]


# ---------------------------------------------------------------------------
# textures
# ---------------------------------------------------------------------------
def _smoothstep_matrix(n_out: int, period: float, n_lat: int) -> np.ndarray:
    """Dense [n_out, n_lat] matrix that interpolates a periodic 1-D lattice
    (spacing ``period`` texels) at texel centres with smoothstep weights."""
    t = (np.arange(n_out, dtype=np.float64) + 0.5) / period
    i0 = np.floor(t).astype(np.int64)
    f = t - i0
    s = f * f * (3.0 - 2.0 * f)
    m = np.zeros((n_out, n_lat), dtype=np.float64)
    rows = np.arange(n_out)
    np.add.at(m, (rows, i0 % n_lat), 1.0 - s)
    np.add.at(m, (rows, (i0 + 1) % n_lat), s)
    return m


def value_noise(height: int, width: int, period: float, octaves: int, gain: float,
                rng: np.random.Generator) -> np.ndarray:
    """Multi-octave value noise in [0, 1] (lattice values U[0,1], smoothstep
    interpolation, period halving and amplitude x``gain`` per octave)."""
    out = np.zeros((height, width), dtype=np.float64)
    amp, total = 1.0, 0.0
    p = float(period)
    for _ in range(octaves):
        p = max(p, 1.0)
        ny = max(2, int(math.ceil(height / p)))
        nx = max(2, int(math.ceil(width / p)))
        lat = rng.random((ny, nx))
        my = _smoothstep_matrix(height, p, ny)
        mx = _smoothstep_matrix(width, p, nx)
        out += amp * (my @ lat @ mx.T)
        total += amp
        amp *= gain
        p *= 0.5
    return out / total


def synthetic_texture(width: int, height: int, channels: int, seed: int,
                      n_base: int = 4, octaves: int = 5, gain: float = 0.5,
                      detail: float = 0.1) -> np.ndarray:
    """A ``height x width x channels`` float32 texture set in [0, 1].

    ``n_base`` smooth value-noise base fields (base period = side/8) are mixed
    into every channel with random convex weights, plus ``detail`` of an
    independent fine value-noise field per channel; each channel is then
    rescaled to [0, 1].  Channels are therefore a low-rank mix, like the
    material texture sets of the paper's evaluation data.
    """
    rng = np.random.default_rng(seed)
    base_period = max(2.0, min(width, height) / 8.0)
    base = [value_noise(height, width, base_period, octaves, gain, rng) for _ in range(n_base)]
    tex = np.empty((height, width, channels), dtype=np.float32)
    for c in range(channels):
        w = rng.random(n_base) + 0.05
        w /= w.sum()
        f = sum(wi * b for wi, b in zip(w, base))
        fine = value_noise(height, width, 4.0, 1, 1.0, rng)
        f = (1.0 - detail) * f + detail * fine
        lo, hi = float(f.min()), float(f.max())
        tex[:, :, c] = ((f - lo) / max(hi - lo, 1e-12)).astype(np.float32)
    return tex


def box_mip_chain_u8(tex: np.ndarray) -> list[np.ndarray]:
    """8-bit reference mip chain: mip 0 is ``tex`` rounded to u8, every further
    mip a 2x2 box average of the float level above it (down to 1x1), each
    level rounded to u8 on its own.  Stands in for the dataset's 8-bit
    sources and Lanczos chain (App. I)."""
    levels = []
    cur = tex.astype(np.float64)
    while True:
        levels.append(np.clip(np.rint(cur * 255.0), 0, 255).astype(np.uint8))
        h, w = cur.shape[:2]
        if h == 1 and w == 1:
            break
        h2, w2 = max(1, h // 2), max(1, w // 2)
        if h > 1 and w > 1:
            cur = cur.reshape(h2, 2, w2, 2, -1).mean(axis=(1, 3))
        elif h > 1:
            cur = cur.reshape(h2, 2, w, -1).mean(axis=1)
        else:
            cur = cur.reshape(h, w2, 2, -1).mean(axis=2)
    return levels


# ---------------------------------------------------------------------------
# latent grids and MLP initial values
# ---------------------------------------------------------------------------
def uniform_grid_values(shape, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    """float32 grid values uniform in [lo, hi]."""
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def random_mlp(k_in: int, hidden: int, c_out: int, seed: int, n_used: int | None = None,
               gain: float = 1.0, hidden_layers: int = 2):
    """Linear layers ``k_in -> hidden -> hidden [-> hidden] -> c_out`` (two or
    three hidden layers) initialised U(+-gain/sqrt(fan_in)), weights stored
    ``[out][in]`` (float32).  Columns of the first layer at or beyond
    ``n_used`` (the zero padding of the input row) are set to zero.  Returns
    ``[w1, b1, w2, b2, (wm, bm,) w3, b3]`` in layer order."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = [(k_in, hidden)] + [(hidden, hidden)] * (hidden_layers - 1) + [(hidden, c_out)]
    for fi, fo in shapes:
        fan = n_used if (fi == k_in and n_used) else fi
        bound = gain / math.sqrt(fan)
        w = rng.uniform(-bound, bound, size=(fo, fi)).astype(np.float32)
        b = rng.uniform(-bound, bound, size=(fo,)).astype(np.float32)
        out += [w, b]
    if n_used is not None and n_used < k_in:
        out[0][:, n_used:] = 0.0
    return out


# ---------------------------------------------------------------------------
# queries
# ---------------------------------------------------------------------------
def random_queries(n: int, mips: int, seed: int, lod_max: int | None = None) -> np.ndarray:
    """``[n, 3]`` float32 rows (u, v, lod): u, v uniform in [0, 1), lod an
    integer uniform over 0 .. ``lod_max`` (default: mips-1)."""
    rng = np.random.default_rng(seed)
    hi = (mips - 1) if lod_max is None else lod_max
    q = np.empty((n, 3), dtype=np.float32)
    q[:, 0] = rng.random(n, dtype=np.float32)
    q[:, 1] = rng.random(n, dtype=np.float32)
    q[:, 2] = rng.integers(0, hi + 1, size=n).astype(np.float32)
    # float32 rounding can push a value to exactly 1.0; keep [0, 1)
    np.minimum(q[:, :2], np.float32(1.0 - 2.0 ** -24), out=q[:, :2])
    return q


def random_texel_queries(width: int, height: int, mips: int, n: int, seed: int) -> np.ndarray:
    """``[n, 3]`` float32 rows (u, v, lod) placed exactly at texel centres of a
    random integer mip level (lod uniform over 0..mips-1)."""
    rng = np.random.default_rng(seed)
    m = rng.integers(0, mips, size=n)
    wm = np.maximum(1, width >> m)
    hm = np.maximum(1, height >> m)
    x = (rng.random(n) * wm).astype(np.int64)
    y = (rng.random(n) * hm).astype(np.int64)
    q = np.empty((n, 3), dtype=np.float32)
    q[:, 0] = (x + 0.5) / wm
    q[:, 1] = (y + 0.5) / hm
    q[:, 2] = m
    return q


def camera_queries(px_w: int, px_h: int, tex_side: int, mips: int,
                   height: float = 1.5, pitch_deg: float = 60.0, hfov_deg: float = 90.0,
                   uv_per_unit: float = 0.25, stride: int = 1):
    """Screen queries of a pinhole camera over a textured ground plane.

    The camera sits ``height`` units above the plane z = 0, its view axis
    tilted ``pitch_deg`` away from straight down, ``hfov_deg`` horizontal
    field of view.  The plane carries texture coordinates
    ``uv = uv_per_unit * (X, Y)``, repeated (wrapped to [0, 1)).  Per pixel
    the continuous level of detail is ``log2(max(|duv/dx|, |duv/dy|) *
    tex_side)`` from the analytic screen-space derivatives (one pixel step),
    clamped to ``[0, mips-1]``.

    Returns float32 ``[n, 3]`` rows (u, v, lambda) for every ``stride``-th
    pixel in row-major order, with ``n = ceil(px_h*px_w/stride)``.
    """
    idx = np.arange(0, px_w * px_h, stride, dtype=np.int64)
    py = (idx // px_w).astype(np.float64)
    px = (idx % px_w).astype(np.float64)
    th = math.tan(math.radians(hfov_deg) / 2.0)
    aspect = px_h / px_w
    pitch = math.radians(pitch_deg)
    fwd = np.array([0.0, math.sin(pitch), -math.cos(pitch)])
    right = np.array([1.0, 0.0, 0.0])
    up = np.cross(right, fwd)

    def hit(sx, sy):
        nx = (2.0 * (sx + 0.5) / px_w - 1.0) * th
        ny = (1.0 - 2.0 * (sy + 0.5) / px_h) * th * aspect
        d = fwd[None, :] + nx[:, None] * right[None, :] + ny[:, None] * up[None, :]
        dz = np.minimum(d[:, 2], -1e-6)
        t = height / (-dz)
        return uv_per_unit * t * d[:, 0], uv_per_unit * t * d[:, 1]

    u0, v0 = hit(px, py)
    u1, v1 = hit(px + 1.0, py)
    u2, v2 = hit(px, py + 1.0)
    dx = np.hypot(u1 - u0, v1 - v0)
    dy = np.hypot(u2 - u0, v2 - v0)
    lam = np.log2(np.maximum(np.maximum(dx, dy) * tex_side, 1e-30))
    lam = np.clip(lam, 0.0, mips - 1.0)
    q = np.empty((idx.size, 3), dtype=np.float32)
    q[:, 0] = np.mod(u0, 1.0)
    q[:, 1] = np.mod(v0, 1.0)
    q[:, 2] = lam
    np.minimum(q[:, :2], np.float32(1.0 - 2.0 ** -24), out=q[:, :2])
    return q


def material_set_shapes(n: int, seed: int, log2_lo: int = 8, log2_hi: int = 12,
                        channel_choices=(8, 12, 16)):
    """Shapes of a batch of ``n`` square materials: side ``2**k`` with k
    uniform over ``log2_lo..log2_hi`` (log-uniform sides snapped to powers of
    two) and a channel count drawn uniformly from ``channel_choices``.
    Returns a list of ``(side, channels)``."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(log2_lo, log2_hi + 1, size=n)
    cs = rng.choice(np.asarray(channel_choices), size=n)
    return [(1 << int(k), int(c)) for k, c in zip(ks, cs)]
