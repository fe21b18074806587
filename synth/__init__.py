"""Seeded synthetic inputs for the sort workloads.

This module holds no sorting arithmetic: it only draws keys.  It is the one
module shared by the tests, the benchmark and the smoke check; both the CPU
oracle and the CUDA library receive its arrays as plain inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used
as a counter-based generator: the i-th draw for a seed is

    x_i = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15  mod 2^64)

(the i-th output of the sequential SplitMix64 stream started at ``seed``),
and u_i = x_i >> 32 is the 32-bit draw.  Every function exists twice, in
numpy (host, used by tests) and in torch (any device, used for large
benchmark inputs); the tests check that both give the same bits.

Distributions (the paper measured uniform keys only, Section 5; the rest
follow the distribution suite of the randomized sample sort study the paper
compares against):
  uniform      u_i
  gaussian     floor((u_{4i} + u_{4i+1} + u_{4i+2} + u_{4i+3}) / 4)
  zero         0
  sorted       the uniform keys sorted ascending
  reverse      the uniform keys sorted descending
  bucket       p = 128 chunks; chunk c, group g = (i mod (n/p)) div (n/p^2):
               key = (g << 25) | (u_i >> 7)
  staggered    chunk c holds range r = (2c + 1) mod p: key = (r << 25) | (u_i >> 7)
float32 keys map each uint32 key u monotonically to
  f = float(int32(u ^ 0x80000000) >> 8) * 2^-23  in [-1, 1)   (exact),
except the zero distribution, which is +0.0f.
Pairs: value = original index; keys either Zipf(1.1) over 2^10 distinct
values or u_i & 0xF0000000 (16 distinct values).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

DISTRIBUTIONS = ("uniform", "gaussian", "zero", "sorted", "reverse",
                 "bucket", "staggered")
P_CHUNKS = 128


def seed_for(config: int, dist: int, rep: int = 0) -> int:
    """Fixed seed per (config, distribution, repetition)."""
    return (10024464 << 16) + (config << 8) + dist + (rep << 48)


# ---------------------------------------------------------------- numpy side

def _mix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def draws64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """x_i for i in [start, start + n) as uint64 (numpy)."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
    return _mix64_np(z)


def draws32(seed: int, n: int, start: int = 0) -> np.ndarray:
    return (draws64(seed, n, start) >> np.uint64(32)).astype(np.uint32)


def keys_u32(dist: str, n: int, seed: int) -> np.ndarray:
    """uint32 keys of one distribution (numpy)."""
    if dist == "uniform":
        return draws32(seed, n)
    if dist == "gaussian":
        u = draws32(seed, 4 * n).astype(np.uint64).reshape(n, 4)
        return (u.sum(axis=1) >> np.uint64(2)).astype(np.uint32)
    if dist == "zero":
        return np.zeros(n, np.uint32)
    if dist == "sorted":
        return np.sort(draws32(seed, n))
    if dist == "reverse":
        return np.sort(draws32(seed, n))[::-1].copy()
    if dist in ("bucket", "staggered"):
        u = draws32(seed, n)
        i = np.arange(n, dtype=np.int64)
        chunk = max(1, n // P_CHUNKS)
        c = np.minimum(i // chunk, P_CHUNKS - 1)
        if dist == "bucket":
            group_len = max(1, chunk // P_CHUNKS)
            r = np.minimum((i % chunk) // group_len, P_CHUNKS - 1)
        else:
            r = (2 * c + 1) % P_CHUNKS
        return ((r.astype(np.uint32) << np.uint32(25)) | (u >> np.uint32(7))).astype(np.uint32)
    raise ValueError("unknown distribution %r" % dist)


def u32_to_f32(u: np.ndarray, zero: bool = False) -> np.ndarray:
    """Monotone exact map of uint32 draws to float32 in [-1, 1)."""
    if zero:
        return np.zeros(u.shape, np.float32)
    s = (u ^ np.uint32(0x80000000)).view(np.int32) >> 8
    return (s.astype(np.float32) * np.float32(2.0 ** -23)).astype(np.float32)


def keys_f32(dist: str, n: int, seed: int) -> np.ndarray:
    return u32_to_f32(keys_u32(dist, n, seed), zero=(dist == "zero"))


def zipf_table(n_distinct: int = 1024, s_exp: float = 1.1) -> np.ndarray:
    """CDF of P(k) ~ k^-s, k = 1..n_distinct, accumulated in fixed order."""
    w = np.arange(1, n_distinct + 1, dtype=np.float64) ** (-s_exp)
    cdf = np.cumsum(w)
    return cdf / cdf[-1]


def keys_zipf(n: int, seed: int, n_distinct: int = 1024, s_exp: float = 1.1) -> np.ndarray:
    """Zipf(s_exp) keys over n_distinct distinct uint32 values."""
    x = draws64(seed, n)
    unit = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    cdf = zipf_table(n_distinct, s_exp)
    rank = np.minimum(np.searchsorted(cdf, unit, side="right"), n_distinct - 1)
    values = draws32(seed ^ 0xA5A5A5A5A5A5A5A5, n_distinct)
    return values[rank]


def keys_16distinct(n: int, seed: int) -> np.ndarray:
    return draws32(seed, n) & np.uint32(0xF0000000)


def batch_sizes(num: int, seed: int, lo_log2: int = 7, hi_log2: int = 20,
                cap: int = 1 << 30) -> np.ndarray:
    """Sizes of the arrays of a batched workload, log-uniform in
    [2^lo, 2^hi]: size_k = floor(2^(lo + (hi - lo) x_k)) with x_k =
    (x_k64 >> 11) * 2^-53 in [0, 1).  If they sum to more than cap, every
    size is scaled by one factor f (floor(size * f), at least 2^lo), f the
    largest of cap/sum, cap/sum * (1 - 2^-10), ... that keeps the sum <= cap."""
    x = (draws64(seed, num) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    sizes = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * x)).astype(np.int64)
    total = int(sizes.sum())
    if total <= cap:
        return sizes
    f = cap / total
    while True:
        scaled = np.maximum(np.floor(sizes * f).astype(np.int64), 1 << lo_log2)
        if int(scaled.sum()) <= cap:
            return scaled
        f *= 1.0 - 2.0 ** -10


def keys_u64(n: int, seed: int) -> np.ndarray:
    return draws64(seed, n)


def keys_zipf_u64(n: int, seed: int) -> np.ndarray:
    """64-bit Zipf(1.1) keys over 2^10 distinct values: the 32-bit Zipf key z
    in the high word, z ^ 0x9E3779B9 in the low word."""
    z = keys_zipf(n, seed).astype(np.uint64)
    return (z << np.uint64(32)) | (z ^ np.uint64(0x9E3779B9))


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate: sums
    of exponential gaps -ln(1 - x_k) / rate, x_k = (x_k64 >> 11) * 2^-53."""
    x = (draws64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.cumsum(-np.log1p(-x) / rate)


# ---------------------------------------------------------------- torch side

def _mix64_t(z):
    import torch
    # logical right shift on int64 storage: arithmetic shift, then mask
    def shr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)
    m1 = torch.tensor(M1 - (1 << 64), dtype=torch.int64, device=z.device)
    m2 = torch.tensor(M2 - (1 << 64), dtype=torch.int64, device=z.device)
    z = (z ^ shr(z, 30)) * m1
    z = (z ^ shr(z, 27)) * m2
    return z ^ shr(z, 31)


def draws64_torch(seed: int, n: int, device="cpu", start: int = 0):
    """x_i as int64 bit patterns (torch, any device)."""
    import torch
    i = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    g = GAMMA - (1 << 64)
    sd = seed & MASK64
    sd = sd - (1 << 64) if sd >= (1 << 63) else sd
    z = i * g + sd
    return _mix64_t(z)


def draws32_torch(seed: int, n: int, device="cpu", start: int = 0):
    """u_i as int64 values in [0, 2^32) (torch)."""
    x = draws64_torch(seed, n, device, start)
    return (x >> 32) & 0xFFFFFFFF


def _to_u32_storage(v):
    """int64 values in [0, 2^32) -> torch.int32 tensor with the same bits."""
    import torch
    v = torch.where(v >= (1 << 31), v - (1 << 32), v)
    return v.to(torch.int32)


def keys_u32_torch(dist: str, n: int, seed: int, device="cpu"):
    """uint32 keys (bit patterns in a torch.int32 tensor) of one distribution."""
    import torch
    if dist == "uniform":
        return _to_u32_storage(draws32_torch(seed, n, device))
    if dist == "gaussian":
        u = draws32_torch(seed, 4 * n, device).view(n, 4)
        return _to_u32_storage(u.sum(dim=1) >> 2)
    if dist == "zero":
        return torch.zeros(n, dtype=torch.int32, device=device)
    if dist in ("sorted", "reverse"):
        u = draws32_torch(seed, n, device)
        v = torch.sort(u, descending=(dist == "reverse")).values
        return _to_u32_storage(v)
    if dist in ("bucket", "staggered"):
        u = draws32_torch(seed, n, device)
        i = torch.arange(n, dtype=torch.int64, device=device)
        chunk = max(1, n // P_CHUNKS)
        c = torch.clamp(i // chunk, max=P_CHUNKS - 1)
        if dist == "bucket":
            group_len = max(1, chunk // P_CHUNKS)
            r = torch.clamp((i % chunk) // group_len, max=P_CHUNKS - 1)
        else:
            r = (2 * c + 1) % P_CHUNKS
        return _to_u32_storage((r << 25) | (u >> 7))
    raise ValueError("unknown distribution %r" % dist)


def keys_f32_torch(dist: str, n: int, seed: int, device="cpu"):
    """float32 keys (torch.float32) of one distribution."""
    import torch
    if dist == "zero":
        return torch.zeros(n, dtype=torch.float32, device=device)
    u = keys_u32_torch(dist, n, seed, device).to(torch.int64) & 0xFFFFFFFF
    s = ((u ^ 0x80000000) & 0xFFFFFFFF)
    s = torch.where(s >= (1 << 31), s - (1 << 32), s) >> 8
    return s.to(torch.float32) * (2.0 ** -23)
