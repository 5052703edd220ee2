"""The benchmark workloads at their full stated sizes, every output compared
with the CPU oracle byte for byte (zero tolerance: with b >= M there is at
most one renormalization per symbol, so the interleaved stream does not depend
on how many lanes run at once and the oracle's stream is the only correct
one, Sections 3 and 5).

  * 1 GiB in 16384 chunks of 64 Ki symbols, 32 coders per chunk: every chunk,
    the header and the offset table, in the launch configuration the
    benchmark times (rans_encode, rans_decode).
  * 4096 binary streams of 64 Ki symbols with per-stream p0: every stream's
    message, in the layout the benchmark's autotuner picks.
  * 10,000 streams of log-uniform size 1 KiB..16 MiB with per-stream
    Dirichlet(0.3) models: every stream's message, autotuned layout, one
    persistent launch each way.
  * a serving trace with request sizes log-uniform 4 KiB..64 MiB and
    per-request Dirichlet(0.5) models over 64..256 symbols: every result.

The oracle runs on all host cores (one stream or chunk per task); its calls
release the interpreter lock.  Inputs come from the seeded generators the
benchmark uses (paper_1402_3392_b300.workloads)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1402_3392_b300 import autotune
from paper_1402_3392_b300 import batch as B
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def cores():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


def test_chunked_1GiB_every_chunk_equals_oracle(rlib, orc, cuda):
    import torch

    cfg = wl.WORKLOADS["chunked"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    n, N, CS = cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    d = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), cuda)
    msg, _, _ = rlib.encode(d, freq, N, CS)
    out, _ = rlib.decode(msg, n, freq, N, CS)
    assert torch.equal(out, d)
    del out
    h_msg = msg.cpu().numpy()
    h_sym = d.cpu().numpy()
    n_chunks = n // CS
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    h = h_msg[:32].view(np.uint32)
    assert list(h[:4]) == [0x534E4152, 1, N, 12]
    assert int(h[4]) | (int(h[5]) << 32) == n and list(h[6:8]) == [CS, n_chunks]
    offs = h_msg[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)

    def check(c):
        ref = orc.encode_chunk(h_sym[c * CS:(c + 1) * CS], freq, N=N)
        got = h_msg[data0 + offs[c]:data0 + offs[c + 1]]
        return got.size == ref.size and np.array_equal(got, ref)

    with ThreadPoolExecutor(cores()) as ex:
        ok = list(ex.map(check, range(n_chunks)))
    bad = [c for c, v in enumerate(ok) if not v]
    assert not bad, bad[:10]
    # offsets start at 0 and the message ends at the last chunk, padded to 16
    # bytes with zeros
    assert offs[0] == 0
    assert h_msg.size == data0 + (offs[-1] + 15) // 16 * 16
    assert not h_msg[data0 + offs[-1]:].any()
    assert not h_msg[32 + 4 * (n_chunks + 1):data0].any()


def _streams_vs_oracle(orc, eb, sym_arena, sym_offs, sizes, tables, table_of, N, cs,
                       group_bytes=1 << 31):
    """Compare every stream's message in an EncodedBatch with the oracle's,
    groups of streams at a time (bounded host memory).  Returns the indices
    of the streams that differ."""
    msg_sizes = eb.host_sizes()
    bad = []
    i = 0
    count = len(sizes)
    while i < count:
        j, acc = i, 0
        while j < count and (j == i or acc + sizes[j] <= group_bytes):
            acc += int(sizes[j])
            j += 1
        s0, s1 = int(sym_offs[i]), int(sym_offs[j - 1]) + int(sizes[j - 1])
        m0, m1 = int(eb.offsets[i]), int(eb.offsets[j - 1]) + int(msg_sizes[j - 1])
        h_sym = sym_arena[s0:s1].cpu().numpy()
        h_msg = eb.arena[m0:m1].cpu().numpy()

        def check(k):
            sym = h_sym[int(sym_offs[k]) - s0:int(sym_offs[k]) - s0 + int(sizes[k])]
            ref = orc.encode_message(sym, tables[table_of[k]], N=int(N[k]),
                                     chunk_symbols=int(cs[k]))
            got = h_msg[int(eb.offsets[k]) - m0:int(eb.offsets[k]) - m0 + int(msg_sizes[k])]
            return got.size == ref.size and np.array_equal(got, ref)

        order = sorted(range(i, j), key=lambda k: -int(sizes[k]))  # largest first
        with ThreadPoolExecutor(cores()) as ex:
            for k, v in zip(order, ex.map(check, order)):
                if not v:
                    bad.append(k)
        del h_sym, h_msg
        i = j
    return sorted(bad)


def test_binary_4096_streams_every_stream_equals_oracle(rlib, orc, cuda):
    """The binary workload as the benchmark runs it: the autotuner's layout
    (tuned on all the streams), batched encode, batched decode."""
    import torch

    cfg = wl.WORKLOADS["binary"]
    count = cfg["n_chunks"]
    per = cfg["n_symbols"] // count
    rng = wl.rng_for("binary")
    p0 = wl.binary_chunk_probs(rng, count, cfg["p0_lo"], cfg["p0_hi"])
    tables = [rlib.rans_quantize_table(wl.weights_from_probs(np.array([p, 1.0 - p]))) for p in p0]
    sizes = np.full(count, per, dtype=np.int64)
    offs, arena_bytes = B.aligned_offsets(sizes)
    probs = [np.array([p, 1.0 - p]) for p in p0]
    sym = wl.streams_on_device(probs, sizes, offs, arena_bytes, wl.seed_for("binary"), cuda)
    tdev = B.upload_tables(tables, cuda)
    idx = np.arange(count)
    best, _ = autotune.autotune(sym, offs, sizes, tdev, idx, widths=(32,), reps=2)
    cs = autotune.chunk_sizes(sizes, best["chunk"], best["policy"])
    eb = B.encode_batch(sym, offs, sizes, tdev, idx, 32, cs)
    torch.cuda.synchronize()
    assert not eb.status.any()
    bad = _streams_vs_oracle(orc, eb, sym, offs, sizes, tables, idx, np.full(count, 32), cs)
    assert not bad, (best, bad[:10])
    dec = B.BatchDecoder(eb.arena, eb.offsets, eb.host_sizes(), sizes, tdev, idx, 32, cs,
                         out_offsets=offs,
                         out_arena=torch.zeros(arena_bytes, dtype=torch.uint8, device=cuda))
    dec()
    torch.cuda.synchronize()
    assert not dec.status.any()
    assert torch.equal(dec.out_arena, sym)


def test_batched_10000_streams_every_stream_equals_oracle(rlib, orc, cuda):
    """The 10,000-stream workload as the benchmark runs it (same draw, the
    autotuner's layout on the same sample of every 25th stream): every
    stream's message equals the oracle's, and one persistent decode launch
    returns every stream's symbols."""
    import torch

    cfg = wl.WORKLOADS["batched"]
    count = cfg["n_streams"]
    rng = wl.rng_for("batched")
    sizes = wl.log_uniform_sizes(rng, count, cfg["size_lo"], cfg["size_hi"])
    probs = wl.batched_models(rng, count, cfg["alpha_lo"], cfg["alpha_hi"], cfg["dirichlet"])
    tables = [rlib.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    offs, arena_bytes = B.aligned_offsets(sizes)
    arena = wl.streams_on_device(probs, sizes, offs, arena_bytes, wl.seed_for("batched"), cuda)
    tdev = B.upload_tables(tables, cuda)
    idx = np.arange(count)
    sample = np.arange(0, count, 25)
    best, _ = autotune.autotune(arena, offs[sample], sizes[sample], tdev, sample, reps=2)
    N = best["n_lanes"]
    cs = autotune.chunk_sizes(sizes, best["chunk"], best["policy"])
    eb = B.encode_batch(arena, offs, sizes, tdev, idx, N, cs)
    torch.cuda.synchronize()
    assert not eb.status.any()
    eb._keep = None
    bad = _streams_vs_oracle(orc, eb, arena, offs, sizes, tables, idx, np.full(count, N), cs)
    assert not bad, (best, bad[:10])
    dec = B.BatchDecoder(eb.arena, eb.offsets, eb.host_sizes(), sizes, tdev, idx, N, cs,
                         out_offsets=offs,
                         out_arena=torch.zeros(arena_bytes, dtype=torch.uint8, device=cuda))
    dec()
    torch.cuda.synchronize()
    assert not dec.status.any()
    assert torch.equal(dec.out_arena, arena)


def test_serving_full_size_trace_every_result_equals_oracle(rlib, orc, cuda):
    """A Poisson trace of 64 encode and decode requests (50/50) with sizes
    log-uniform 4 KiB..64 MiB and per-request Dirichlet(0.5) models over
    64..256 symbols, in the benchmark's layout (N = 32, 64 Ki-symbol chunks),
    served from a 4 GiB device budget with host payloads: every encode result
    equals the oracle's message and every decode result the symbols the
    oracle's message holds."""
    import ctypes

    import torch

    cfg = wl.WORKLOADS["serving"]
    count, N, CS = 64, 32, 1 << 16
    rng = np.random.default_rng(wl.seed_for("serving", 3))
    sizes = wl.log_uniform_sizes(rng, count, cfg["size_lo"], cfg["size_hi"])
    probs = wl.batched_models(rng, count, cfg["alpha_lo"], cfg["alpha_hi"], cfg["dirichlet"])
    tables = [rlib.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    kinds = rng.integers(0, 2, size=count)
    arrivals = wl.poisson_arrivals(rng, 2000.0, count)
    syms = [wl.iid_symbols(rng, p, int(n)) for p, n in zip(probs, sizes)]
    with ThreadPoolExecutor(cores()) as ex:
        msgs = list(ex.map(lambda k: orc.encode_message(syms[k], tables[k], N=N, chunk_symbols=CS),
                           range(count)))
    reqs = np.zeros(count, dtype=rlib.REQUEST_DTYPE)
    keep, expect = [], []
    for i in range(count):
        if kinds[i] == rlib.RANS_REQ_ENCODE:
            inp, exp, cap = syms[i], msgs[i], rlib.rans_max_encoded_size(syms[i].size, N, CS)
        else:
            inp, exp, cap = msgs[i], syms[i], syms[i].size
        h_in = torch.from_numpy(inp).pin_memory()
        h_out = torch.zeros(max(cap, 1), dtype=torch.uint8).pin_memory()
        keep += [h_in, h_out]
        expect.append(exp)
        reqs[i] = (kinds[i], i, N, CS, h_in.data_ptr(), inp.size, syms[i].size, h_out.data_ptr(),
                   cap, arrivals[i])
    tdev = B.upload_tables(tables, cuda)
    budget = torch.empty(4 << 30, dtype=torch.uint8, device=cuda)
    srv = rlib.Server(tdev, budget, max_batch=16, n_slots=3)
    res = srv.run(reqs)
    srv.close()
    assert (res["status"] == 0).all(), res["status"]
    for i in range(count):
        n_out = int(res["output_size"][i])
        got = np.ctypeslib.as_array((ctypes.c_uint8 * max(n_out, 1)).from_address(
            int(reqs["output"][i])))[:n_out]
        assert n_out == expect[i].size and np.array_equal(got, expect[i]), (i, int(kinds[i]))
    assert sizes.max() > (16 << 20) and sizes.min() < (64 << 10)   # the trace spans the range
