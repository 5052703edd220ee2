"""Binary models (symbols 0 and 1, f_0 + f_1 = M, both > 0: rABS in the
paper's terms, Section 2) are decoded without a slot table: the symbol is
[slot >= f_0] and D two multiply-adds.  The bitstream is the plain one, so
the oracle's Algorithm-1 coder is the reference: every message is compared
byte for byte, every decode symbol for symbol, through the single-message
and the batched entry points, at the extreme frequencies, with partial
steps, ragged last chunks, odd chunk counts (a warp's second chunk missing)
and models that switch between binary and not from stream to stream."""
import zlib

import numpy as np
import pytest

from paper_1402_3392_b300 import batch as B
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def binary_table(f0):
    f = np.zeros(2, dtype=np.uint16)
    f[0], f[1] = f0, 4096 - f0
    return f


def draw(rng, f, n):
    return (rng.random(n) >= f[0] / 4096.0).astype(np.uint8)


@pytest.mark.parametrize("f0", [1, 2, 977, 2048, 3500, 4094, 4095])
@pytest.mark.parametrize("N,CS", [(32, 65536), (32, 4096), (7, 1000), (1, 333)])
def test_single_message_binary_matches_oracle(rlib, orc, cuda, f0, N, CS):
    import torch

    rng = np.random.default_rng(zlib.crc32(repr((f0, N, CS)).encode()))
    f = binary_table(f0)
    n = 3 * CS + CS // 3 + 5
    sym = draw(rng, f, n)
    d = torch.from_numpy(sym).to(cuda)
    msg, _, _ = rlib.encode(d, f, N, CS)
    ref = orc.encode_message(sym, f, N=N, chunk_symbols=CS)
    assert np.array_equal(msg.cpu().numpy(), ref)
    out, _ = rlib.decode(torch.from_numpy(ref).to(cuda), n, f, N, CS)
    assert np.array_equal(out.cpu().numpy(), sym)


def test_binary_model_listed_with_trailing_zeros(rlib, orc, cuda):
    """A 256-entry table with f_2.. = 0 is the same binary model."""
    import torch

    rng = np.random.default_rng(5)
    f = np.zeros(256, dtype=np.uint16)
    f[0], f[1] = 3000, 1096
    sym = draw(rng, f, 100_001)
    ref = orc.encode_message(sym, f, N=32, chunk_symbols=8192)
    out, _ = rlib.decode(torch.from_numpy(ref).to(cuda), sym.size, f, 32, 8192)
    assert np.array_equal(out.cpu().numpy(), sym)


def test_batched_binary_and_other_models_interleaved(rlib, orc, cuda):
    """Streams alternate between binary models, a three-symbol model and a
    256-symbol one, so the batched decoder's CTAs switch between the
    table-free step and the slot table from item to item; chunk counts are
    odd (pairs with one chunk missing) and tails ragged."""
    import torch

    rng = np.random.default_rng(211)
    tables, streams = [], []
    for i in range(48):
        k = i % 4
        if k in (0, 1):
            f = binary_table(int(rng.integers(1, 4096)))
        elif k == 2:
            f = rlib.rans_quantize_table(wl.weights_from_probs(np.array([0.6, 0.3, 0.1])))
        else:
            f = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
        tables.append(f)
        n = int(rng.integers(1, 200_000))
        sym = rng.choice(len(f), size=n, p=f / f.sum()).astype(np.uint8)
        CS = int(rng.choice([4096, 5000, 16384, 65536]))
        N = int(rng.choice([32, 32, 9]))
        streams.append(dict(sym=sym, table=i, N=N, CS=CS))
    msgs = [orc.encode_message(s["sym"], tables[s["table"]], N=s["N"], chunk_symbols=s["CS"])
            for s in streams]
    offs, total = B.aligned_offsets([m.size for m in msgs])
    host = np.zeros(total, dtype=np.uint8)
    for m, o in zip(msgs, offs):
        host[o:o + m.size] = m
    arena = torch.from_numpy(host).to(cuda)
    dec = B.BatchDecoder(arena, offs, [m.size for m in msgs], [s["sym"].size for s in streams],
                         B.upload_tables(tables, cuda), [s["table"] for s in streams],
                         [s["N"] for s in streams], [s["CS"] for s in streams])
    status = dec()
    torch.cuda.synchronize()
    assert not status.any(), status.cpu().numpy()
    for i, s in enumerate(streams):
        assert np.array_equal(dec.output(i).cpu().numpy(), s["sym"]), i
    # and the batched encoder's messages are the oracle's
    sym_offs, sym_total = B.aligned_offsets([s["sym"].size for s in streams])
    sh = np.zeros(max(sym_total, B.ALIGN), dtype=np.uint8)
    for s, o in zip(streams, sym_offs):
        sh[o:o + s["sym"].size] = s["sym"]
    eb = B.encode_batch(torch.from_numpy(sh).to(cuda), sym_offs, [s["sym"].size for s in streams],
                        B.upload_tables(tables, cuda), [s["table"] for s in streams],
                        [s["N"] for s in streams], [s["CS"] for s in streams])
    torch.cuda.synchronize()
    assert not eb.status.any()
    for i, m in enumerate(msgs):
        assert np.array_equal(eb.message(i).cpu().numpy(), m), i


def test_damaged_binary_batch_stream_is_reported(rlib, orc, cuda):
    """A binary stream whose data bytes were rewritten fails alone with
    RANS_ERR_CORRUPT when the oracle rejects it too; its neighbours decode."""
    import torch

    import oracle

    rng = np.random.default_rng(223)
    f = binary_table(3100)
    syms = [draw(rng, f, 70_000) for _ in range(3)]
    msgs = [orc.encode_message(s, f, N=32, chunk_symbols=16384) for s in syms]
    bad = msgs[1].copy()
    bad[-40:-20] ^= 0x5A
    with pytest.raises(oracle.OracleError):
        orc.decode_message(bad, syms[1].size, f, N=32, chunk_symbols=16384)
    msgs[1] = bad
    offs, total = B.aligned_offsets([m.size for m in msgs])
    host = np.zeros(total, dtype=np.uint8)
    for m, o in zip(msgs, offs):
        host[o:o + m.size] = m
    dec = B.BatchDecoder(torch.from_numpy(host).to(cuda), offs, [m.size for m in msgs],
                         [s.size for s in syms], B.upload_tables([f], cuda), 0, 32, 16384)
    st = dec().cpu().numpy()
    assert list(st) == [0, rlib.RANS_ERR_CORRUPT, 0]
    for i in (0, 2):
        assert np.array_equal(dec.output(i).cpu().numpy(), syms[i])


def test_batched_binary_edge_streams(rlib, orc, cuda):
    """In one batch: an empty binary stream (its header is still checked), a
    binary-looking table that is not a valid model (f_0 + f_1 = M plus one
    more symbol: RANS_ERR_INVALID_ARG for that stream alone), one-chunk and
    odd-chunk binary streams, and a 256-symbol stream."""
    import torch

    rng = np.random.default_rng(227)
    good = binary_table(2900)
    bad = np.zeros(256, dtype=np.uint16)
    bad[0], bad[1], bad[7] = 2900, 1196, 3
    zipf = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
    tables = [good, bad, zipf]
    plan = [(0, 0), (0, 5000), (0, 3 * 4096 + 17), (1, 9000), (2, 30_000), (0, 1)]
    syms, msgs = [], []
    for t, n in plan:
        f = tables[t] if t != 1 else good            # the bad table's message is a good one
        s = draw(rng, f, n) if t != 2 else rng.choice(256, size=n, p=zipf / zipf.sum()).astype(np.uint8)
        syms.append(s)
        msgs.append(orc.encode_message(s, f, N=32, chunk_symbols=4096))
    offs, total = B.aligned_offsets([m.size for m in msgs])
    host = np.zeros(total, dtype=np.uint8)
    for m, o in zip(msgs, offs):
        host[o:o + m.size] = m
    dec = B.BatchDecoder(torch.from_numpy(host).to(cuda), offs, [m.size for m in msgs],
                         [s.size for s in syms], B.upload_tables(tables, cuda),
                         [t for t, _ in plan], 32, 4096)
    st = dec().cpu().numpy()
    assert list(st) == [0, 0, 0, rlib.RANS_ERR_INVALID_ARG, 0, 0]
    for i in (1, 2, 4, 5):
        assert np.array_equal(dec.output(i).cpu().numpy(), syms[i]), i


def test_batched_binary_encode_edge_streams(rlib, orc, cuda):
    """The batched encoder codes binary-model streams as warp items (one
    chunk a warp, the model's two entries in registers): in one batch with a
    256-symbol stream, an empty binary stream gets its header-only message,
    one-chunk and ragged ones the oracle's bytes, a binary-looking table that
    is not a valid model (f_0 + f_1 = M plus one more symbol) fails alone
    with RANS_ERR_INVALID_ARG, and a symbol outside {0, 1} in a binary
    stream with RANS_ERR_ZERO_FREQ (size 0)."""
    import torch

    rng = np.random.default_rng(229)
    good = binary_table(2900)
    bad = np.zeros(256, dtype=np.uint16)
    bad[0], bad[1], bad[7] = 2900, 1196, 3
    zipf = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
    tables = [good, bad, zipf]
    plan = [(0, 0, 32), (0, 5000, 32), (0, 3 * 4096 + 17, 32), (1, 9000, 32), (2, 30_000, 32),
            (0, 1, 32), (0, 7000, 32), (0, 2 * 4096 + 5, 11)]
    syms = []
    for t, n, _ in plan:
        if t == 2:
            syms.append(rng.choice(256, size=n, p=zipf / zipf.sum()).astype(np.uint8))
        else:
            syms.append(draw(rng, good, n))
    syms[6][3333] = 2  # not a symbol of the binary model
    offs, total = B.aligned_offsets([s.size for s in syms])
    host = np.zeros(max(total, B.ALIGN), dtype=np.uint8)
    for s, o in zip(syms, offs):
        host[o:o + s.size] = s
    eb = B.encode_batch(torch.from_numpy(host).to(cuda), offs, [s.size for s in syms],
                        B.upload_tables(tables, cuda), [t for t, _, _ in plan],
                        [n for _, _, n in plan], 4096)
    torch.cuda.synchronize()
    st = eb.status.cpu().numpy()
    want = [0, 0, 0, rlib.RANS_ERR_INVALID_ARG, 0, 0, rlib.RANS_ERR_ZERO_FREQ, 0]
    assert list(st) == want
    sizes = eb.host_sizes()
    for i, (t, _, N) in enumerate(plan):
        if want[i]:
            assert sizes[i] == 0, i
            continue
        ref = orc.encode_message(syms[i], tables[t], N=N, chunk_symbols=4096)
        assert np.array_equal(eb.message(i).cpu().numpy(), ref), i
