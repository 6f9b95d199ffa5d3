"""Gaussian test matrices G for the randomized steps of randUTV (Fig. 4).

Counter layout (one Philox4x32-10 call per pair of rows):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (r div 2, c, step, index)
for row r (0-based, within the active block) and column c of the k x b matrix
G drawn at global step ``step`` (1-based, as in Fig. 4); ``index`` is the
matrix's position in a batch (0 for a single matrix).  Words (x0, x1) and
(x2, x3) become two uniforms u1, u2 on the open interval (0, 1) from the top
52 bits of each 64-bit word pair, u = (floor(w / 2^12) + 1/2) 2^-52, which
is exact in FP64 and lies in [2^-53, 1 - 2^-53]; the Box-Muller pair
  z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2)
fills row 2p with z0 and row 2p+1 with z1.

The batched FP32 form draws from the same words with 23-bit uniforms
u = (floor(x / 2^9) + 1/2) 2^-23 of words x1 (u1) and x3 (u2), exact in FP32;
``step_gaussian_f32`` is that definition evaluated in FP64 and rounded once.
"""
import numpy as np
from .philox import philox4x32_10

_TWO_M52 = 2.0 ** -52


def uniform52(lo, hi):
    """Map two uint32 words (lo, hi) to ((hi*2^32 + lo) >> 12 + 0.5) * 2^-52 in (0, 1)."""
    w = (np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * _TWO_M52


def step_words(seed, step, k, b, index=0):
    """Raw Philox words for step ``step``: four uint32 arrays of shape (ceil(k/2), b)."""
    p = np.arange((k + 1) // 2, dtype=np.uint64)[:, None]
    c = np.arange(b, dtype=np.uint64)[None, :]
    seed = int(seed)
    return philox4x32_10(p, c, np.uint64(step), np.uint64(index), seed & 0xFFFFFFFF, seed >> 32)


def step_gaussian(seed, step, k, b, index=0):
    """The k x b Gaussian matrix G of global step ``step`` (float64, shape (k, b))."""
    x0, x1, x2, x3 = step_words(seed, step, k, b, index)
    u1 = uniform52(x0, x1)
    u2 = uniform52(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    g = np.empty(((k + 1) // 2 * 2, b))
    g[0::2] = r * np.cos(t)
    g[1::2] = r * np.sin(t)
    return g[:k]


def uniform23(x):
    """(floor(x / 2^9) + 1/2) 2^-23 for uint32 words x: exact in FP32, in (0, 1)."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def step_gaussian_f32(seed, step, k, b, index=0):
    """G of the batched FP32 form (matrix ``index``, step ``step``), float32
    (k, b): Box-Muller on the 23-bit uniforms of words x1, x3, in FP64, rounded."""
    x0, x1, x2, x3 = step_words(seed, step, k, b, index)
    u1 = uniform23(x1)
    u2 = uniform23(x3)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    g = np.empty(((k + 1) // 2 * 2, b))
    g[0::2] = r * np.cos(t)
    g[1::2] = r * np.sin(t)
    return g[:k].astype(np.float32)


def stream_layout(m, n, b, p=0):
    """(step, k, offset) for every step of an m x n factorization with block b
    that draws a Gaussian, i.e. steps i with b*i < min(m, n) (both I3 and J3
    non-empty in Fig. 4).  ``offset`` counts doubles in the concatenated stream
    where step i's k x (b+p) matrix is stored column-major (leading dimension k)."""
    out, off, i = [], 0, 1
    while b * i < min(m, n):
        k = m - b * (i - 1)
        out.append((i, k, off))
        off += k * (b + p)
        i += 1
    return out, off


def gaussian_stream(seed, m, n, b, p=0):
    """All steps' G concatenated column-major in the layout of ``stream_layout``."""
    layout, total = stream_layout(m, n, b, p)
    buf = np.empty(total)
    w = b + p
    for step, k, off in layout:
        buf[off:off + k * w] = step_gaussian(seed, step, k, w).ravel(order="F")
    return buf
