"""Host-side marshalling for the batched entry points (rans_encode_batch,
rans_decode_batch): device arenas, descriptor arrays and model tables.

Nothing here touches the data: the coding runs in the CUDA kernels behind the
C ABI.  An "arena" is one torch uint8 device buffer that many streams' inputs
or outputs live in, each at a 256-byte aligned offset, so that a batch of
thousands of streams needs one allocation and one descriptor upload.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import rans

ALIGN = 256


def aligned_offsets(sizes, align: int = ALIGN):
    """Offsets of consecutive regions of the given sizes, each aligned."""
    sizes = np.asarray(sizes, dtype=np.int64)
    padded = (np.maximum(sizes, 1) + align - 1) // align * align
    offs = np.zeros(sizes.size, dtype=np.int64)
    if sizes.size > 1:
        offs[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum()) if sizes.size else 0
    return offs, total


def upload_tables(tables, device):
    """Model tables (sequence of <=256 u16 frequencies each) as a device
    array of [n_tables, 256] u16 (zero padded)."""
    import torch

    arr = np.zeros((len(tables), 256), dtype=np.uint16)
    for i, f in enumerate(tables):
        f = np.asarray(f, dtype=np.uint16)
        arr[i, :f.size] = f
    return torch.from_numpy(arr.view(np.int16)).to(device)


def _per_stream(v, n, dtype=np.int64):
    a = np.asarray(v, dtype=dtype)
    return np.full(n, a, dtype=dtype) if a.ndim == 0 else a


@dataclass
class EncodedBatch:
    arena: object            # torch uint8 device buffer holding every message
    offsets: np.ndarray      # message offsets in the arena
    caps: np.ndarray         # capacity reserved per message
    sizes: object            # device u64 per stream (message sizes)
    status: object           # device u32 per stream
    n_symbols: np.ndarray
    table: np.ndarray
    n_lanes: np.ndarray
    chunk_symbols: np.ndarray

    def host_sizes(self) -> np.ndarray:
        return self.sizes.cpu().numpy().astype(np.int64)

    def message(self, i: int):
        size = int(self.sizes[i].item())
        o = int(self.offsets[i])
        return self.arena[o:o + size]


def encode_batch(sym_arena, sym_offsets, n_symbols, tables_dev, table, n_lanes=32,
                 chunk_symbols=65536, stream=None, out_arena=None, scratch=None):
    """Encode streams whose symbols lie in sym_arena at sym_offsets.  Returns
    an EncodedBatch (asynchronous: sizes/status are device tensors)."""
    import torch

    dev = sym_arena.device
    n = len(n_symbols)
    n_symbols = np.asarray(n_symbols, dtype=np.int64)
    table = _per_stream(table, n, np.int64)
    n_lanes = _per_stream(n_lanes, n, np.int64)
    chunk_symbols = _per_stream(chunk_symbols, n, np.int64)
    caps = np.array([rans.rans_max_encoded_size(int(a), int(b), int(c))
                     for a, b, c in zip(n_symbols, n_lanes, chunk_symbols)], dtype=np.int64)
    offs, total = aligned_offsets(caps)
    if out_arena is None:
        out_arena = torch.empty(max(total, ALIGN), dtype=torch.uint8, device=dev)
    d = np.zeros(n, dtype=rans.ENCODE_STREAM_DTYPE)
    d["symbols"] = sym_arena.data_ptr() + np.asarray(sym_offsets, dtype=np.int64)
    d["n_symbols"] = n_symbols
    d["out"] = out_arena.data_ptr() + offs
    d["out_cap"] = caps
    d["table"] = table
    d["n_lanes"] = n_lanes
    d["chunk_symbols"] = chunk_symbols
    scap = rans.rans_encode_batch_plan(d)
    if scratch is None or scratch.numel() < scap:
        scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    d_desc = torch.from_numpy(d.view(np.uint8).copy()).to(dev)
    sizes = torch.zeros(n, dtype=torch.int64, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    rans.rans_encode_batch(d_desc, n, tables_dev, tables_dev.shape[0], sizes, status, scratch,
                           scratch.numel(), stream)
    eb = EncodedBatch(out_arena, offs, caps, sizes, status, n_symbols, table, n_lanes,
                      chunk_symbols)
    eb._keep = (d_desc, scratch)
    return eb


def decode_descriptors(msg_ptrs, msg_sizes, out_ptrs, n_symbols, table, n_lanes, chunk_symbols):
    n = len(n_symbols)
    d = np.zeros(n, dtype=rans.STREAM_DTYPE)
    d["msg"] = msg_ptrs
    d["msg_size"] = msg_sizes
    d["symbols"] = out_ptrs
    d["n_symbols"] = n_symbols
    d["table"] = _per_stream(table, n)
    d["n_lanes"] = _per_stream(n_lanes, n)
    d["chunk_symbols"] = _per_stream(chunk_symbols, n)
    return d


class BatchDecoder:
    """Decode many messages with one rans_decode_batch call.  Descriptors
    and scratch are uploaded/allocated once, so the call can be repeated or
    captured in a CUDA graph."""

    def __init__(self, msg_arena, msg_offsets, msg_sizes, n_symbols, tables_dev, table,
                 n_lanes=32, chunk_symbols=65536, out_arena=None, out_offsets=None):
        import torch

        dev = msg_arena.device
        n = len(n_symbols)
        self.n = n
        self.n_symbols = np.asarray(n_symbols, dtype=np.int64)
        if out_arena is None:
            out_offsets, total = aligned_offsets(self.n_symbols)
            out_arena = torch.empty(max(total, ALIGN), dtype=torch.uint8, device=dev)
        self.out_arena, self.out_offsets = out_arena, np.asarray(out_offsets, dtype=np.int64)
        desc = decode_descriptors(msg_arena.data_ptr() + np.asarray(msg_offsets, dtype=np.int64),
                                  np.asarray(msg_sizes, dtype=np.int64),
                                  out_arena.data_ptr() + self.out_offsets, self.n_symbols, table,
                                  n_lanes, chunk_symbols)
        self.d_desc = torch.from_numpy(desc.view(np.uint8).copy()).to(dev)
        self.tables = tables_dev
        self.status = torch.zeros(n, dtype=torch.int32, device=dev)
        scap = rans.rans_decode_batch_scratch_size(n)
        self.scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
        self._msg_arena = msg_arena

    def __call__(self, stream=None):
        rans.rans_decode_batch(self.d_desc, self.n, self.tables, self.tables.shape[0],
                               self.status, self.scratch, self.scratch.numel(), stream)
        return self.status

    def output(self, i: int):
        o = int(self.out_offsets[i])
        return self.out_arena[o:o + int(self.n_symbols[i])]
