"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws input data.  It holds none of the method's
arithmetic, so both the CUDA library's tests and the oracle can be fed from
it.  Every generator is a pure function of its arguments (numpy PCG64 seeded
by ``seed``) and returns ``(X, Q)``: the data set and held-out queries drawn
from the same distribution, both float32, row-major.

* :func:`gaussian_mixture` -- isotropic clusters (the tiny case).
* :func:`mnist_like`       -- 28 x 28 stroke images with integer pixel values
  0..255 and about 80 % zeros; stands in for MNIST (Table II: n = 60,000,
  d = 784), which is not available here.
* :func:`lognormal_int`    -- heavy-tailed non-negative integers 0..255 per
  dimension; stands in for SIFT-like descriptors (d = 128).
* :func:`latent_factor`    -- [0, 1] values from rank-64 latent factors plus
  noise; stands in for GIST-like descriptors (d = 960).
* :func:`unit_gaussian`    -- the paper's fully specified "Random" set:
  N(0, I) vectors normalised to unit length (Sec. IV-A).
* :func:`uneven_batches`   -- a stream of batch sizes (log-uniform in
  1..4096) with per-batch k and v draws.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_mixture(n: int, d: int, m: int, n_centres: int = 100, sigma: float = 0.3,
                     seed: int = 0):
    """Mixture of ``n_centres`` isotropic Gaussians, centres ~ N(0, I),
    per-cluster standard deviation ``sigma``; n points plus m queries."""
    g = _rng(seed)
    centres = g.standard_normal((n_centres, d))
    lab = g.integers(0, n_centres, size=n + m)
    pts = centres[lab] + sigma * g.standard_normal((n + m, d))
    pts = pts.astype(np.float32)
    return np.ascontiguousarray(pts[:n]), np.ascontiguousarray(pts[n:])


def _segment_distance(px, py, ax, ay, bx, by):
    """Distance from pixel centres (px, py) to the segment a-b (broadcast)."""
    vx, vy = bx - ax, by - ay
    wx, wy = px - ax, py - ay
    den = vx * vx + vy * vy + 1e-9
    t = np.clip((wx * vx + wy * vy) / den, 0.0, 1.0)
    cx, cy = ax + t * vx - px, ay + t * vy - py
    return np.sqrt(cx * cx + cy * cy)


def mnist_like(n: int, m: int, n_prototypes: int = 60, side: int = 28, seed: int = 0,
               chunk: int = 4096):
    """Stroke images on a side x side grid (d = side^2), integer values 0..255.

    Each prototype is a random 4-segment polyline in the central region with
    a base stroke width.  A sample takes a prototype, jitters its control
    points (N(0, 1.1 px)), shifts it by up to 2 px (control points stay at
    least 4 px inside the grid), scales the stroke width
    by U(0.8, 1.3) and rasterises: pixels within the stroke core are 255, a
    one-pixel ramp gives intermediate grey values, everything else 0 (about
    80 % of the pixels).  The border is almost always blank: a stroke reaches
    it only when a control point sits at the clamp limit with a wide stroke
    (about 0.1 % of images).
    """
    g = _rng(seed)
    total = n + m
    n_ctrl = 5
    lo, hi = 7.0, side - 8.0
    proto = g.uniform(lo, hi, size=(n_prototypes, n_ctrl, 2))
    base_w = g.uniform(1.9, 2.7, size=n_prototypes)
    lab = g.integers(0, n_prototypes, size=total)
    jitter = g.normal(0.0, 1.1, size=(total, n_ctrl, 2))
    shift = g.integers(-2, 3, size=(total, 1, 2)).astype(np.float64)
    wscale = g.uniform(0.8, 1.3, size=total)
    ctrl = np.clip(proto[lab] + jitter + shift, 4.0, side - 5.0)
    width = base_w[lab] * wscale
    yy, xx = np.meshgrid(np.arange(side, dtype=np.float64) + 0.5,
                         np.arange(side, dtype=np.float64) + 0.5, indexing="ij")
    px = xx.reshape(1, -1)
    py = yy.reshape(1, -1)
    out = np.empty((total, side * side), dtype=np.float32)
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        c = ctrl[s:e]
        dist = np.full((e - s, side * side), np.inf)
        for seg in range(n_ctrl - 1):
            ax, ay = c[:, seg, 0:1], c[:, seg, 1:2]
            bx, by = c[:, seg + 1, 0:1], c[:, seg + 1, 1:2]
            dist = np.minimum(dist, _segment_distance(px, py, ax, ay, bx, by))
        w = width[s:e, None]
        val = np.clip(w + 0.5 - dist, 0.0, 1.0) * 255.0
        out[s:e] = np.rint(val).astype(np.float32)
    return np.ascontiguousarray(out[:n]), np.ascontiguousarray(out[n:])


def lognormal_int(n: int, d: int, m: int, seed: int = 0, chunk: int = 1 << 18):
    """Per-dimension log-normal, mu_j ~ U(1, 4), sigma_j ~ U(0.5, 1.5);
    x = clip(round(exp(N(mu_j, sigma_j))), 0, 255)."""
    g = _rng(seed)
    mu = g.uniform(1.0, 4.0, size=d)
    sd = g.uniform(0.5, 1.5, size=d)
    total = n + m
    out = np.empty((total, d), dtype=np.float32)
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        z = g.standard_normal((e - s, d)) * sd + mu
        out[s:e] = np.clip(np.rint(np.exp(z)), 0, 255).astype(np.float32)
    return np.ascontiguousarray(out[:n]), np.ascontiguousarray(out[n:])


def latent_factor(n: int, d: int, m: int, rank: int = 64, seed: int = 0,
                  chunk: int = 1 << 16):
    """x = clip(0.5 + 0.15 (u V^T)/sqrt(rank) + N(0, 0.05^2), 0, 1) with
    u ~ N(0, I_rank) per row and V ~ N(0, 1) (d x rank) shared."""
    g = _rng(seed)
    V = g.standard_normal((d, rank)).astype(np.float32)
    total = n + m
    out = np.empty((total, d), dtype=np.float32)
    scale = np.float32(0.15 / np.sqrt(rank))
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        u = g.standard_normal((e - s, rank)).astype(np.float32)
        noise = g.standard_normal((e - s, d)).astype(np.float32) * np.float32(0.05)
        out[s:e] = np.clip(np.float32(0.5) + scale * (u @ V.T) + noise, 0.0, 1.0)
    return np.ascontiguousarray(out[:n]), np.ascontiguousarray(out[n:])


def unit_gaussian(n: int, d: int, m: int, seed: int = 0):
    """N(0, I) vectors normalised to unit length (Sec. IV-A "Random")."""
    g = _rng(seed)
    pts = g.standard_normal((n + m, d))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    pts = pts.astype(np.float32)
    return np.ascontiguousarray(pts[:n]), np.ascontiguousarray(pts[n:])


def uneven_batches(total: int, max_batch: int = 4096, ks=(1, 10, 100), vs=(2, 5, 8),
                   seed: int = 0):
    """Batch sizes floor(exp(U(0, ln(max_batch + 1)))) clamped to
    [1, max_batch] until ``total`` queries are covered; k and v drawn per
    batch.  Returns a list of (size, k, v)."""
    g = _rng(seed)
    out = []
    done = 0
    while done < total:
        b = int(np.floor(np.exp(g.uniform(0.0, np.log(max_batch + 1)))))
        b = max(1, min(max_batch, b, total - done))
        out.append((b, int(g.choice(ks)), int(g.choice(vs))))
        done += b
    return out
