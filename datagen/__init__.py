"""Seeded synthetic key generators shaped like the paper's workloads.

This module holds input generation only, none of the sorting method's
arithmetic; it is the one module shared by the CPU oracle's tests and the
CUDA path's tests and benchmark.  Every generator takes an explicit integer
seed and draws from numpy's PCG64 bit generator, so the same seed gives the
same bytes on the same numpy build (floating-point transforms go through the
platform's libm, so bytes may differ across machines; parity is always
checked on one machine's bytes).

Datasets (arxiv 2307.08637, Sec. 5 "Synthetic Datasets"):
  uniform01      U[0,1)                       (parity workload, 2^20 keys)
  normal         N(0, 1)
  lognormal      LogN(mu=0, sigma=0.5)
  exponential    Exp(lambda=2)
  chisquared     chi^2(k=4)
  mix_gauss      5 Gaussians, means U[-10,10], sigmas U[0.1,2], equal weights
  uniform_1e6    U[0, 1e6)
  zipf           Zipf(s=0.75) over 1..1e6 (u64), i.i.d. so already shuffled
  root_dups      A[i] = i mod floor(sqrt(N))   (u64, shuffled)
  two_dups       A[i] = (i^2 + N/2) mod N      (u64, shuffled)
  skewed_u64     99% piecewise-linear CDF over 64 equal-width pieces of
                 [0, 2^64) with Dirichlet(0.3) masses + 1% in 100 tight
                 lognormal(sigma=2) clusters (u64)
The paper's real-world datasets are not available; these stand in for its
synthetic suite only.
"""
from __future__ import annotations

import numpy as np

F64_DISTS = ("normal", "lognormal", "exponential", "chisquared", "mix_gauss", "uniform_1e6")
U64_DUP_DISTS = ("zipf", "root_dups", "two_dups")
ALL_DISTS = ("uniform01",) + F64_DISTS + U64_DUP_DISTS + ("skewed_u64",)


def _rng(seed: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFFFFFFFFFF, salt]))


def _zipf_table(nvals: int, s: float) -> np.ndarray:
    w = np.arange(1, nvals + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def generate(dist: str, n: int, seed: int) -> np.ndarray:
    """n keys of distribution `dist` (float64 or uint64 per the list above)."""
    n = int(n)
    g = _rng(seed, 1 + ALL_DISTS.index(dist) if dist in ALL_DISTS else 99)
    if dist == "uniform01":
        return g.random(n)
    if dist == "normal":
        return g.standard_normal(n)
    if dist == "lognormal":
        return g.lognormal(0.0, 0.5, n)
    if dist == "exponential":
        return g.exponential(1.0 / 2.0, n)
    if dist == "chisquared":
        return g.chisquare(4.0, n)
    if dist == "mix_gauss":
        means = g.uniform(-10.0, 10.0, 5)
        sig = g.uniform(0.1, 2.0, 5)
        comp = g.integers(0, 5, n)
        return means[comp] + sig[comp] * g.standard_normal(n)
    if dist == "uniform_1e6":
        return g.uniform(0.0, 1e6, n)
    if dist == "zipf":
        table = _zipf_table(1_000_000, 0.75)
        u = g.random(n)
        return (np.searchsorted(table, u, side="right") + 1).astype(np.uint64)
    if dist == "root_dups":
        m = int(np.floor(np.sqrt(n))) if n > 0 else 1
        a = (np.arange(n, dtype=np.uint64) % np.uint64(max(m, 1)))
        return a[g.permutation(n)]
    if dist == "two_dups":
        i = np.arange(n, dtype=np.uint64)
        nn = np.uint64(max(n, 1))
        a = ((i * i) % nn + np.uint64(n // 2)) % nn
        return a[g.permutation(n)]
    if dist == "skewed_u64":
        return _skewed_u64(g, n)
    raise KeyError(dist)


def _skewed_u64(g: np.random.Generator, n: int) -> np.ndarray:
    nclu = n // 100
    nmain = n - nclu
    masses = g.dirichlet(np.full(64, 0.3))
    piece = g.choice(64, size=nmain, p=masses)
    width = 2.0 ** 58
    # within a piece the density is linear: draw the offset by inverting a
    # linear density whose slope is random per piece
    slope = g.uniform(-1.0, 1.0, 64)[piece]
    u = g.random(nmain)
    # inverse CDF of f(t) = 1 + slope (2t - 1) on [0, 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = slope
        t = np.where(np.abs(a) < 1e-9, u,
                     ((a - 1.0) + np.sqrt((1.0 - a) ** 2 + 4.0 * a * u)) / (2.0 * a))
    t = np.clip(t, 0.0, np.nextafter(1.0, 0.0))
    main = (piece.astype(np.uint64) << np.uint64(58)) + (t * width).astype(np.uint64)
    centers = g.integers(0, 2 ** 63, size=100, dtype=np.uint64) * np.uint64(2) + g.integers(0, 2, size=100,
                                                                                            dtype=np.uint64)
    c = g.integers(0, 100, size=nclu)
    off = np.floor(g.lognormal(0.0, 2.0, nclu)).astype(np.uint64)
    base = centers[c]
    clu = base + off
    clu = np.where(clu < base, np.uint64(0xFFFFFFFFFFFFFFFF), clu)  # saturate
    out = np.concatenate([main, clu])
    return out[g.permutation(n)]


def segment_lengths(nseg: int, seed: int, lo: float = 1e3, hi: float = 1e6) -> np.ndarray:
    """Segment lengths floor(exp(U[ln lo, ln hi])) (log-uniform)."""
    g = _rng(seed, 1000)
    return np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), nseg))).astype(np.int64)


def segmented(nseg: int, seed: int, lo: float = 1e3, hi: float = 1e6,
              dists: tuple = F64_DISTS) -> tuple[np.ndarray, np.ndarray, list]:
    """Batched workload: nseg float64 arrays, log-uniform lengths in [lo, hi],
    each from a distribution picked uniformly from `dists`, shifted by
    U[-1e3, 1e3] and scaled by a log-uniform factor in [1e-3, 1e3].
    Returns (keys, offsets[nseg+1], per-segment distribution names)."""
    lens = segment_lengths(nseg, seed, lo, hi)
    g = _rng(seed, 2000)
    pick = g.integers(0, len(dists), nseg)
    shift = g.uniform(-1e3, 1e3, nseg)
    scale = np.exp(g.uniform(np.log(1e-3), np.log(1e3), nseg))
    off = np.zeros(nseg + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens).astype(np.uint64)
    keys = np.empty(int(off[-1]), dtype=np.float64)
    names = []
    for s in range(nseg):
        d = dists[pick[s]]
        names.append(d)
        x = generate(d, int(lens[s]), seed * 1_000_003 + s)
        keys[int(off[s]):int(off[s + 1])] = shift[s] + scale[s] * x
    return keys, off, names


def skewed_u64_device(n: int, seed: int, device: str = "cuda:0"):
    """The skewed u64 workload generated on a GPU (for 2e9 keys, where the
    numpy generator above would take minutes), as an int64 tensor holding
    the u64 bit patterns.  Same recipe, not the same bytes:
      * 64 equal-width pieces of [0, 2^64) with Dirichlet(0.3) masses and a
        random linear density per piece (slope in [-1, 1]); the offset inside
        a piece comes from inverting that density in FP32, which fixes its
        top 24 bits, and the remaining 34 bits are uniform;
      * each position is, with probability 1/100, a cluster key instead:
        center + floor(LogN(0, 2)), saturating, 100 uniform u64 centers.
    Piece masses, slopes and centers are drawn with numpy from `seed`; the
    per-key draws use a torch generator seeded from it."""
    import torch

    g = _rng(seed, 3000)
    masses = g.dirichlet(np.full(64, 0.3))
    slope_np = g.uniform(-1.0, 1.0, 64)
    centers_np = g.integers(0, 2 ** 63, size=100, dtype=np.uint64) * np.uint64(2) + \
        g.integers(0, 2, size=100, dtype=np.uint64)
    tg = torch.Generator(device=device)
    tg.manual_seed(int(g.integers(0, 2 ** 62)))
    cdf = torch.tensor(np.cumsum(masses), dtype=torch.float64, device=device)
    cdf[-1] = 1.0
    slope = torch.tensor(slope_np, dtype=torch.float32, device=device)
    centers = torch.tensor(centers_np.view(np.int64), device=device)
    out = torch.empty(n, dtype=torch.int64, device=device)
    step = 1 << 27
    for a in range(0, n, step):
        m = min(step, n - a)
        u_piece = torch.rand(m, generator=tg, device=device, dtype=torch.float64)
        piece = torch.searchsorted(cdf, u_piece, right=True).clamp_(max=63)
        del u_piece
        s = slope[piece]
        u = torch.rand(m, generator=tg, device=device, dtype=torch.float32)
        # inverse CDF of f(t) = 1 + s (2t - 1) on [0, 1)
        disc = torch.sqrt(torch.clamp((1.0 - s) ** 2 + 4.0 * s * u, min=0.0))
        t = torch.where(s.abs() < 1e-6, u, ((s - 1.0) + disc) / (2.0 * s)).clamp_(0.0, 0.99999994)
        del s, u, disc
        top = (t * 16777216.0).to(torch.int64)  # 24 bits
        low = torch.randint(0, 1 << 34, (m,), generator=tg, device=device, dtype=torch.int64)
        key = (piece.to(torch.int64) << 58) | (top << 34) | low
        del t, top, low, piece
        clu = torch.rand(m, generator=tg, device=device, dtype=torch.float32) < 0.01
        k = int(clu.sum())
        if k:
            c = torch.randint(0, 100, (k,), generator=tg, device=device)
            z = torch.randn(k, generator=tg, device=device, dtype=torch.float32)
            off = torch.floor(torch.exp(2.0 * z)).to(torch.int64)
            base = centers[c]
            # unsigned saturating add on int64 bit patterns: the sum wrapped
            # iff it is below the base in unsigned order
            ssum = base + off
            mn = -(1 << 63)
            wrapped = (ssum ^ mn) < (base ^ mn)
            key[clu] = torch.where(wrapped, torch.full_like(base, -1), ssum)
        out[a:a + m] = key
    return out
