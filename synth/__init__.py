"""Seeded synthetic inputs for the Camelot query pipelines.

This module is shared by the CPU oracle and the CUDA path, so it holds no
arithmetic of the method: it only draws the raw inputs (query images, token
IDs, weights, arrival times, profiling draws).  Every tensor comes from its own
numpy ``PCG64`` stream, derived from ``(seed, tensor tag)`` through
``numpy.random.SeedSequence`` so that adding a tensor never shifts another.

Value distributions follow the workloads the paper evaluates with
(Sec. 3, Table 1 stand-ins):

* query images: uniform uint8 in [0, 255], HWC layout;
* dense weights: N(0, 1/fan_in), row-major ``[out, in]``, drawn in float64 and
  rounded once to float32 (the reduced-precision arms round these again);
* text queries: token IDs Zipf(s) over the vocabulary, length uniform in
  ``[lo, hi]``;
* arrivals: Poisson process (exponential gaps) at a given rate, or the
  sinusoidal (diurnal) rate used for the low-load policy (Sec. 8.2-8.3).
"""
from __future__ import annotations

import zlib

import numpy as np

__all__ = [
    "rng", "images_u8", "dense_weights", "mlp_weights", "zipf_tokens",
    "poisson_arrivals_ns", "diurnal_arrivals_ns", "CFG1", "CFG2", "CFG3", "CFG4", "cfg4_inputs",
    "cfg1_inputs", "cfg2_inputs",
]

# Shapes of the synthetic workloads (query pipeline configurations).
CFG1 = dict(n_queries=1024, H=64, W=64, C=3, dims=(12288, 512, 256, 10), batch=16)
CFG2 = dict(H=224, W=224, C=3, dims=(37632, 1024, 1024, 1000), top_k=5, qos_ms=20.0)
CFG3 = dict(dims=(12, 64, 64, 1), n_samples=20000)
CFG4 = dict(vocab=32000, d_model=512, d_ff=2048, n_tags=64, zipf_s=1.1, seq=(16, 128))


def rng(seed: int, tag: str) -> np.random.Generator:
    """Independent generator for tensor ``tag`` under ``seed``."""
    key = zlib.crc32(tag.encode("utf-8")) & 0xFFFFFFFF
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), key])))


def images_u8(seed: int, n: int, H: int, W: int, C: int, tag: str = "images") -> np.ndarray:
    """``n`` images, uniform uint8, shape ``[n, H, W, C]`` (HWC, C-contiguous)."""
    return rng(seed, tag).integers(0, 256, size=(n, H, W, C), dtype=np.uint8)


def dense_weights(seed: int, out_dim: int, in_dim: int, tag: str) -> np.ndarray:
    """Row-major ``[out_dim, in_dim]`` float32 weights ~ N(0, 1/in_dim)."""
    w = rng(seed, tag).standard_normal((out_dim, in_dim)) * (1.0 / np.sqrt(in_dim))
    return w.astype(np.float32)


def mlp_weights(seed: int, dims, tag: str = "mlp") -> list:
    """Weights of a chain ``dims[0] -> dims[1] -> ...``, one matrix per layer."""
    return [dense_weights(seed, dims[i + 1], dims[i], f"{tag}.w{i}") for i in range(len(dims) - 1)]


def zipf_tokens(seed: int, n_queries: int, vocab: int, s: float, lo: int, hi: int,
                tag: str = "tokens"):
    """Token-ID queries: list of int32 arrays, IDs = Zipf rank - 1 over ``vocab``
    ranks (inverse CDF of the truncated Zipf law), lengths uniform in [lo, hi]."""
    g = rng(seed, tag)
    ranks = np.arange(1, vocab + 1, dtype=np.float64)
    pmf = ranks ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    lens = g.integers(lo, hi + 1, size=n_queries)
    out = []
    for L in lens:
        u = g.random(int(L))
        out.append(np.minimum(np.searchsorted(cdf, u, side="right"), vocab - 1).astype(np.int32))
    return out


def poisson_arrivals_ns(seed: int, n: int, rate_qps: float, tag: str = "arrivals") -> np.ndarray:
    """Arrival offsets (int64 ns from 0) of a Poisson process at ``rate_qps``."""
    gaps = rng(seed, tag).exponential(1.0 / rate_qps, size=n)
    t = np.cumsum(gaps) - gaps[0]
    return np.round(t * 1e9).astype(np.int64)


def diurnal_arrivals_ns(seed: int, peak_qps: float, period_s: float, lo_frac: float = 0.10,
                        hi_frac: float = 1.0, tag: str = "diurnal") -> np.ndarray:
    """Non-homogeneous Poisson arrivals over one period with rate
    ``peak*(m - a*cos(2*pi*t/period))`` (minimum ``lo_frac*peak`` at t=0, maximum
    ``hi_frac*peak`` at mid-period), drawn by thinning."""
    g = rng(seed, tag)
    m, a = (hi_frac + lo_frac) / 2.0, (hi_frac - lo_frac) / 2.0
    lam_max = peak_qps * hi_frac
    n_cand = int(lam_max * period_s * 1.2) + 64
    t = np.cumsum(g.exponential(1.0 / lam_max, size=n_cand))
    t = t[t < period_s]
    keep = g.random(t.size) < (m - a * np.cos(2 * np.pi * t / period_s)) / hi_frac
    return np.round(t[keep] * 1e9).astype(np.int64)


def cfg1_inputs(seed: int = 0, n_queries: int = CFG1["n_queries"]):
    """Plain 2-stage pipeline inputs: images ``[n,64,64,3]`` u8 and the three
    MLP weight matrices (12288->512->256->10)."""
    x = images_u8(seed, n_queries, CFG1["H"], CFG1["W"], CFG1["C"], tag="cfg1.images")
    ws = mlp_weights(seed, CFG1["dims"], tag="cfg1")
    return x, ws


def cfg2_inputs(seed: int = 0, n_queries: int = 64):
    """3-stage pipeline inputs: images ``[n,224,224,3]`` u8 and weights
    37632->1024->1024 and 1024->1000 (float32; the BF16 arm rounds them)."""
    x = images_u8(seed, n_queries, CFG2["H"], CFG2["W"], CFG2["C"], tag="cfg2.images")
    ws = mlp_weights(seed, CFG2["dims"], tag="cfg2")
    return x, ws


def cfg4_inputs(seed: int = 0, n_queries: int = 64, seq_max: int = 128):
    """Text-tagging pipeline inputs: token queries padded to ``seq_max`` int32
    IDs (-1 = padding; Zipf s = 1.1 over 32000 IDs, lengths uniform in 16..128),
    their lengths, the embedding table [32000, 512] N(0, 1) and the three weight
    matrices 512->2048->512->64 N(0, 1/fan_in), all float32."""
    c = CFG4
    toks = zipf_tokens(seed, n_queries, c["vocab"], c["zipf_s"], c["seq"][0], c["seq"][1],
                       tag="cfg4.tokens")
    padded = np.full((n_queries, seq_max), -1, np.int32)
    lens = np.array([len(t) for t in toks], np.int32)
    for i, t in enumerate(toks):
        padded[i, : len(t)] = t
    E = rng(seed, "cfg4.embedding").standard_normal((c["vocab"], c["d_model"])).astype(np.float32)
    ws = mlp_weights(seed, (c["d_model"], c["d_ff"], c["d_model"], c["n_tags"]), tag="cfg4")
    return padded, lens, E, ws
