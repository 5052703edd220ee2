"""Seeded synthetic workloads for the interleaved rANS coder.

This module only draws random inputs: symbol probabilities, integer weights,
i.i.d. symbol streams and stream-size mixes.  It holds none of the coder's
arithmetic (no C/D, no renormalization, no quantization), so both the CUDA
path and the CPU oracle can be fed from it.

The paper measures on Calgary/Canterbury files and a Linux tarball with an
order-0 static model (Section 7).  Those files are not available here; i.i.d.
symbols drawn from a fixed distribution are exactly what an order-0 static
model sees, so they stand in for them.

Workloads (sizes and distributions):
  single   : 1 MiB i.i.d. bytes, Zipf(s=1.2) over 256 symbols, one stream
  chunked  : 1 GiB i.i.d. bytes, Zipf(s=1.1) over 256 symbols,
             16384 chunks of 64 KiB, 32-way interleaving
  binary   : 256 MiB of {0,1} symbols in 4096 chunks of 64 KiB, chunk k with
             p0 ~ U[0.5, 0.999]
  batched  : 10,000 streams, sizes log-uniform in [1 KiB, 16 MiB], alphabet
             size uniform in [16, 256], Dirichlet(0.3) probabilities
  serving  : Poisson arrivals, sizes log-uniform in [4 KiB, 64 MiB], alphabet
             size uniform in [64, 256], Dirichlet(0.5) probabilities
  bypass   : 512 Mi i.i.d. bytes of the chunked distribution with raw words
             (bypass coding, 8192 chunks of 64 KiB, 32-way interleaving): symbols
             >= 16 carry one raw 16-bit word, uniform in [0, 2^16)
  adaptive : 256 Mi bits for adaptive per-coder contexts, 4096 chunks of
             64 Ki, 32-way interleaving; P(bit = 0) is piecewise constant over
             segments of 4096 symbols, each segment's p0 ~ U[0.001, 0.999]
  adaptive_n: 256 Mi symbols over 16 for adaptive per-coder models, 4096
             chunks of 64 Ki, 32-way interleaving; the distribution is
             constant over runs of 4096 symbols, Dirichlet(0.5) per run
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x1402339200000000

WORKLOADS = {
    "single": dict(index=0, n_symbols=1 << 20, zipf_s=1.2, alphabet=256, n_lanes=32,
                   chunk_symbols=1 << 20),
    "chunked": dict(index=1, n_symbols=1 << 30, zipf_s=1.1, alphabet=256, n_lanes=32,
                    chunk_symbols=1 << 16),
    "binary": dict(index=2, n_symbols=1 << 28, n_chunks=4096, n_lanes=32,
                   chunk_symbols=1 << 16, p0_lo=0.5, p0_hi=0.999),
    "batched": dict(index=3, n_streams=10_000, size_lo=1 << 10, size_hi=1 << 24,
                    alpha_lo=16, alpha_hi=256, dirichlet=0.3),
    "serving": dict(index=4, size_lo=4 << 10, size_hi=64 << 20, alpha_lo=64,
                    alpha_hi=256, dirichlet=0.5, budget_bytes=40 << 30),
    "bypass": dict(index=5, n_symbols=1 << 29, zipf_s=1.1, alphabet=256, raw_from=16,
                   n_lanes=32, chunk_symbols=1 << 16),
    "adaptive": dict(index=6, n_symbols=1 << 28, n_lanes=32, chunk_symbols=1 << 16,
                     segment=4096, p0_lo=0.001, p0_hi=0.999),
    "adaptive_n": dict(index=7, n_symbols=1 << 28, n_alpha=16, n_lanes=32,
                       chunk_symbols=1 << 16, segment=4096, dirichlet=0.5),
}


def seed_for(workload: str, extra: int = 0) -> int:
    return SEED_BASE + WORKLOADS[workload]["index"] + (extra << 8)


def rng_for(workload: str, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng(seed_for(workload, extra))


def zipf_probs(n: int, s: float) -> np.ndarray:
    """p_k proportional to 1/(k+1)^s, k = 0..n-1 (fp64)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    p = k ** (-s)
    return p / p.sum()


def dirichlet_probs(rng: np.random.Generator, n: int, alpha: float) -> np.ndarray:
    p = rng.dirichlet(np.full(n, alpha, dtype=np.float64))
    # Dirichlet draws with small alpha can underflow to exactly 0; keep every
    # symbol possible so the model covers the alphabet.
    p = np.maximum(p, 1e-300)
    return p / p.sum()


def weights_from_probs(p: np.ndarray) -> np.ndarray:
    """Integer weights w_s = max(1, round-half-even(p_s * 2^32)) as uint64."""
    w = np.rint(np.asarray(p, dtype=np.float64) * float(1 << 32))
    return np.maximum(w, 1).astype(np.uint64)


def iid_symbols(rng: np.random.Generator, p: np.ndarray, n: int) -> np.ndarray:
    """n i.i.d. draws from p by inverse CDF, as uint8 (host)."""
    cdf = np.cumsum(np.asarray(p, dtype=np.float64))
    cdf[-1] = 1.0
    u = rng.random(n)
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(p) - 1).astype(np.uint8)


def iid_symbols_device(p: np.ndarray, n: int, seed: int, device, piece: int = 1 << 26):
    """n i.i.d. draws from p generated on a CUDA device (torch), as uint8.

    Used for the large workloads; generated in pieces to bound temporaries."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed & 0x7FFFFFFFFFFFFFFF)
    cdf = torch.tensor(np.cumsum(np.asarray(p, dtype=np.float64)), dtype=torch.float64,
                       device=device)
    cdf[-1] = 1.0
    out = torch.empty(n, dtype=torch.uint8, device=device)
    for a in range(0, n, piece):
        z = min(n, a + piece)
        u = torch.rand(z - a, generator=g, device=device, dtype=torch.float64)
        idx = torch.searchsorted(cdf, u, right=True).clamp_(max=len(p) - 1)
        out[a:z] = idx.to(torch.uint8)
    return out


def log_uniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Sizes with log(size) uniform on [log lo, log hi], as int64."""
    e = rng.uniform(math.log(lo), math.log(hi), size=count)
    return np.clip(np.exp(e).astype(np.int64), lo, hi)


def binary_chunk_probs(rng: np.random.Generator, n_chunks: int, lo: float = 0.5,
                       hi: float = 0.999) -> np.ndarray:
    """Per-chunk p0 ~ U[lo, hi] for the binary workload (fp64)."""
    return rng.uniform(lo, hi, size=n_chunks)


def drifting_bits(rng: np.random.Generator, n: int, segment: int, lo: float = 0.001,
                  hi: float = 0.999) -> np.ndarray:
    """n bits (uint8 0/1); P(bit = 0) is constant over each run of `segment`
    symbols and drawn U[lo, hi] per run (host)."""
    p0 = rng.uniform(lo, hi, size=max(1, -(-n // segment)))
    u = rng.random(n)
    return (u >= np.repeat(p0, segment)[:n]).astype(np.uint8)


def drifting_bits_device(n: int, segment: int, seed: int, device, lo: float = 0.001,
                         hi: float = 0.999, piece: int = 1 << 26):
    """drifting_bits generated on a CUDA device (torch), in pieces; piece must
    be a multiple of segment."""
    import torch

    assert piece % segment == 0
    g = torch.Generator(device=device)
    g.manual_seed(seed & 0x7FFFFFFFFFFFFFFF)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    for a in range(0, n, piece):
        z = min(n, a + piece)
        n_seg = -(-(z - a) // segment)
        p0 = lo + (hi - lo) * torch.rand(n_seg, generator=g, device=device, dtype=torch.float64)
        u = torch.rand(z - a, generator=g, device=device, dtype=torch.float64)
        out[a:z] = (u >= p0.repeat_interleave(segment)[: z - a]).to(torch.uint8)
    return out


def drifting_symbols(rng: np.random.Generator, n: int, n_alpha: int, segment: int,
                     alpha: float = 0.5) -> np.ndarray:
    """n symbols (uint8 < n_alpha) whose distribution is constant over each
    run of `segment` symbols and drawn Dirichlet(alpha) per run (host)."""
    n_seg = max(1, -(-n // segment))
    out = np.empty(n, dtype=np.uint8)
    for k in range(n_seg):
        a, z = k * segment, min(n, (k + 1) * segment)
        p = rng.dirichlet(np.full(n_alpha, alpha))
        cdf = np.cumsum(p)
        cdf[-1] = 1.0
        out[a:z] = np.minimum(np.searchsorted(cdf, rng.random(z - a), side="right"),
                              n_alpha - 1)
    return out


def drifting_symbols_device(n: int, n_alpha: int, segment: int, seed: int, device,
                            alpha: float = 0.5, piece: int = 1 << 26):
    """drifting_symbols generated on a CUDA device (torch), in pieces; piece
    must be a multiple of segment.  The per-run Dirichlet draws are made as
    normalised Gamma(alpha) variates."""
    import torch

    assert piece % segment == 0
    g = torch.Generator(device=device)
    g.manual_seed(seed & 0x7FFFFFFFFFFFFFFF)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    conc = torch.full((n_alpha,), float(alpha), dtype=torch.float64, device=device)
    for a in range(0, n, piece):
        z = min(n, a + piece)
        n_seg = -(-(z - a) // segment)
        gam = torch._standard_gamma(conc.expand(n_seg, n_alpha).contiguous(), generator=g)
        cdf = torch.cumsum(gam / gam.sum(dim=1, keepdim=True), dim=1)
        cdf[:, -1] = 1.0
        u = torch.rand(n_seg * segment, generator=g, device=device, dtype=torch.float64)
        idx = torch.searchsorted(cdf, u.view(n_seg, segment), right=True).view(-1)[: z - a]
        out[a:z] = idx.clamp_(max=n_alpha - 1).to(torch.uint8)
    return out


def poisson_arrivals(rng: np.random.Generator, rate_per_s: float, count: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def batched_models(rng: np.random.Generator, count: int, alpha_lo: int = 16,
                   alpha_hi: int = 256, dirichlet: float = 0.3):
    """Per-stream probability vectors: alphabet size uniform in
    [alpha_lo, alpha_hi], Dirichlet(dirichlet) probabilities."""
    sizes = rng.integers(alpha_lo, alpha_hi + 1, size=count)
    return [dirichlet_probs(rng, int(a), dirichlet) for a in sizes]


def streams_on_device(probs, n_symbols, offsets, arena_bytes: int, seed: int, device,
                      piece: int = 1 << 27):
    """i.i.d. symbols for many streams at once, on the device.  Stream k has
    n_symbols[k] symbols drawn from probs[k], stored at arena[offsets[k]:].
    One search over the concatenated, shifted CDFs (stream k's CDF + k) maps a
    uniform draw u of stream k (value k + u) to its symbol.  Bytes between
    streams (alignment filler) are zero."""
    import torch

    n = len(probs)
    starts = np.zeros(n, dtype=np.int64)
    cdfs = []
    pos = 0
    for k, p in enumerate(probs):
        c = np.cumsum(np.asarray(p, dtype=np.float64))
        c[-1] = 1.0
        cdfs.append(k + c)
        starts[k] = pos
        pos += c.size
    g = torch.tensor(np.concatenate(cdfs), dtype=torch.float64, device=device)
    start_d = torch.tensor(starts, dtype=torch.int64, device=device)
    alpha_d = torch.tensor([len(p) for p in probs], dtype=torch.int64, device=device)
    begins = torch.tensor(np.asarray(offsets, dtype=np.int64), dtype=torch.int64, device=device)
    ends = begins + torch.tensor(np.asarray(n_symbols, dtype=np.int64), dtype=torch.int64,
                                 device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed & 0x7FFFFFFFFFFFFFFF)
    arena = torch.empty(max(arena_bytes, 1), dtype=torch.uint8, device=device)
    for a in range(0, arena_bytes, piece):
        z = min(arena_bytes, a + piece)
        posn = torch.arange(a, z, dtype=torch.int64, device=device)
        k = torch.searchsorted(ends, posn, right=True).clamp_(max=n - 1)
        u = torch.rand(z - a, generator=gen, device=device, dtype=torch.float64)
        idx = torch.searchsorted(g, k.to(torch.float64) + u, right=True)
        sym = torch.minimum(idx - start_d[k], alpha_d[k] - 1).clamp_(min=0)
        sym = torch.where((posn >= begins[k]) & (posn < ends[k]), sym, 0)
        arena[a:z] = sym.to(torch.uint8)
        del posn, k, u, idx, sym
    return arena
