"""Autotuner for the batched coder: picks the interleave width N and the
chunking policy for a workload by timing rans_encode_batch + rans_decode_batch
on a sample of its streams.

The layout is a property of the bitstream (the encoder fixes N and the chunk
size), so the choice is made before encoding.  Candidates:
  N          : 4, 8, 16, 32 (coders per chunk, which is also the lanes a
               stream takes: the decoder maps one coder to one warp lane, so
               N < 32 leaves lanes idle; a warp never holds two streams)
  chunk      : 16, 32, 64, 128, 256 KiB
  per-stream : "fixed" (every stream uses the chunk size) or "fill" (a stream
               shorter than 16 chunks is cut into up to 16 smaller chunks, at
               least 16 KiB each -- the low end of the candidate list, so no
               chunk but a stream's last is below it -- so that its one work
               item keeps more of the 16 chunk slots of a CTA -- 8 warps x 2
               chunks -- busy)
The score is decoded bytes per second of the batched decoder (median of a few
runs); ties go to the larger chunk.  The chosen policy and the chunk sizes it
gives are reported beside the result.
"""
from __future__ import annotations

import statistics

import numpy as np

from . import batch as B

WIDTHS = (4, 8, 16, 32)
CHUNKS = (16 << 10, 32 << 10, 64 << 10, 128 << 10, 256 << 10)
POLICIES = ("fixed", "fill")
ITEM_CHUNKS = 16       # chunks in one work item of the batched decoder
MIN_FILL_CHUNK = CHUNKS[0]


def chunk_sizes(n_symbols, chunk, policy):
    n = np.asarray(n_symbols, dtype=np.int64)
    if policy == "fixed":
        return np.full(n.size, chunk, dtype=np.int64)
    fill = (n + ITEM_CHUNKS - 1) // ITEM_CHUNKS
    fill = np.maximum((fill + 1023) // 1024 * 1024, MIN_FILL_CHUNK)
    return np.minimum(fill, chunk)


def _time(fn, reps):
    import torch

    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def autotune(sym_arena, sym_offsets, n_symbols, tables_dev, table, widths=WIDTHS,
             chunks=CHUNKS, policies=POLICIES, reps=3):  # noqa: D401
    """Return (best, results): best = dict(n_lanes, chunk, policy); results =
    list of dicts with the measured decode GB/s of every candidate."""
    import torch

    n_symbols = np.asarray(n_symbols, dtype=np.int64)
    total = int(n_symbols.sum())
    results = []
    for policy in policies:
        for chunk in chunks:
            cs = chunk_sizes(n_symbols, chunk, policy)
            for N in widths:
                eb = B.encode_batch(sym_arena, sym_offsets, n_symbols, tables_dev, table, N, cs)
                torch.cuda.synchronize()
                if eb.status.any():
                    continue
                dec = B.BatchDecoder(eb.arena, eb.offsets, eb.host_sizes(), n_symbols, tables_dev,
                                     table, N, cs)
                dec()
                ms = _time(dec, reps)
                results.append(dict(n_lanes=N, chunk=chunk, policy=policy,
                                    decode_gbs=total / (ms * 1e-3) / 1e9))
                del eb, dec
    best = max(results, key=lambda r: (round(r["decode_gbs"], 1), r["chunk"]))
    return dict(n_lanes=best["n_lanes"], chunk=best["chunk"], policy=best["policy"]), results
