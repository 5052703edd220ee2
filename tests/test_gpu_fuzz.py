"""Damaged messages of every kind on the GPU against the CPU oracle.

Valid messages are damaged at random -- bytes of the data region rewritten,
offsets of the offset table changed, whole chunks replaced by random bytes
-- and handed to both decoders.  The verdict must agree: where the oracle
rejects the message the GPU reports RANS_ERR_CORRUPT, and where the oracle
accepts it (the damage left a decodable message) the GPU decodes exactly
the oracle's symbols.  The header and the offset table are checked by the
library before any chunk is touched, and every read of a chunk stays inside
the message, so no damage can take the decoders outside their buffers."""
import zlib

import numpy as np
import pytest

import oracle
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu

N, CS = 7, 1500          # 7 coders, ragged steps; 1500-symbol chunks
N_SYM = 20 * CS + 333    # 21 chunks, the last one short


def message(rlib, orc, kind, rng):
    """(message bytes, oracle decode function, GPU decode function)."""
    import torch

    p = wl.zipf_probs(64, 1.0)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    sym = wl.iid_symbols(rng, p, N_SYM)
    if kind == "plain":
        m = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message(b, N_SYM, freq, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode(d, N_SYM, freq, N, CS, sync=False)  # noqa: E731
    elif kind == "bypass":
        raw_words = (np.arange(64) >= 8).astype(np.uint8)
        raw = rng.integers(0, 1 << 16, size=N_SYM).astype(np.uint16)
        m = orc.encode_message_bypass(sym, raw, freq, raw_words, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message_bypass(b, N_SYM, freq, raw_words, N=N,  # noqa: E731
                                                  chunk_symbols=CS)[0]
        gpu = lambda d: rlib.decode_bypass(d, N_SYM, freq, raw_words, N, CS,  # noqa: E731
                                           sync=False)[0::2]
    elif kind == "bytes":
        m = orc.encode_message_bytes(sym, freq, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message_bytes(b, N_SYM, freq, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode_bytes(d, N_SYM, freq, N, CS, sync=False)  # noqa: E731
    elif kind == "adaptive":
        bits = wl.drifting_bits(rng, N_SYM, 500)
        m = orc.encode_message_adaptive(bits, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message_adaptive(b, N_SYM, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode_adaptive(d, N_SYM, N, CS, sync=False)  # noqa: E731
    elif kind == "binary":             # decoded without a slot table
        pb = np.array([0.8, 0.2])
        fb = rlib.rans_quantize_table(wl.weights_from_probs(pb))
        bits = wl.iid_symbols(rng, pb, N_SYM)
        m = orc.encode_message(bits, fb, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message(b, N_SYM, fb, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode(d, N_SYM, fb, N, CS, sync=False)  # noqa: E731
    elif kind == "adaptive_n":         # per-coder models over 9 symbols
        syms = wl.drifting_symbols(rng, N_SYM, 9, 500, 0.5)
        m = orc.encode_message_adaptive_n(syms, 9, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message_adaptive_n(b, N_SYM, 9, N=N,  # noqa: E731
                                                      chunk_symbols=CS)
        gpu = lambda d: rlib.decode_adaptive_n(d, N_SYM, 9, N, CS, sync=False)  # noqa: E731
    elif kind == "wide14":
        f14 = rlib.rans_quantize_table(wl.weights_from_probs(p), 14)
        m = orc.encode_message(sym, f14, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message(b, N_SYM, f14, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode(d, N_SYM, f14, N, CS, sync=False)  # noqa: E731
    else:
        ln = orc.prefix_lengths(wl.weights_from_probs(p), 12)
        m = orc.encode_message_prefix(sym, ln, N=N, chunk_symbols=CS)
        ref = lambda b: orc.decode_message_prefix(b, N_SYM, ln, N=N, chunk_symbols=CS)  # noqa: E731
        gpu = lambda d: rlib.decode_prefix(d, N_SYM, ln, N, CS, sync=False)  # noqa: E731
    return m, ref, gpu, torch


def damage(m, rng, how):
    b = m.copy()
    n_chunks = -(-N_SYM // CS)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = b[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    if how == "bytes":                       # a few random bytes of the data region
        for _ in range(int(rng.integers(1, 4))):
            b[int(rng.integers(data0, b.size))] = rng.integers(0, 256)
    elif how == "offset":                    # one interior offset moved
        c = int(rng.integers(1, n_chunks))
        offs[c] = np.uint32(max(0, int(offs[c]) + int(rng.integers(-9, 10))))
    else:                                    # one chunk replaced by random bytes
        c = int(rng.integers(0, n_chunks))
        a, z = data0 + int(offs[c]), data0 + int(offs[c + 1])
        b[a:z] = rng.integers(0, 256, size=z - a, dtype=np.uint8)
    return b


@pytest.mark.parametrize("kind", ["plain", "bypass", "bytes", "adaptive", "prefix", "wide14",
                                  "binary", "adaptive_n"])
@pytest.mark.parametrize("how", ["bytes", "offset", "chunk"])
def test_damaged_messages_agree_with_oracle(rlib, orc, cuda, kind, how):
    rng = np.random.default_rng(zlib.crc32(repr(("fuzz", kind, how)).encode()))
    m, ref, gpu, torch = message(rlib, orc, kind, rng)
    accepted = 0
    for _ in range(12):
        bad = damage(m, rng, how)
        try:
            want = ref(bad)
        except oracle.OracleError:
            want = None
        out, st = gpu(torch.from_numpy(bad).to(cuda))
        torch.cuda.synchronize()
        st = int(st.item())
        if want is None:
            assert st == rlib.RANS_ERR_CORRUPT, (kind, how)
        else:
            accepted += 1
            assert st == rlib.RANS_OK, (kind, how)
            assert np.array_equal(out.cpu().numpy(), want), (kind, how)
    assert accepted < 12          # the damage was seen at least once


def _gpu_status(torch, gpu, bad, cuda):
    out, st = gpu(torch.from_numpy(bad).to(cuda))
    torch.cuda.synchronize()
    return out, int(st.item())


@pytest.mark.parametrize("kind", ["plain", "bypass", "bytes", "adaptive", "prefix", "wide14",
                                  "binary", "adaptive_n"])
def test_truncated_messages_agree_with_oracle(rlib, orc, cuda, kind):
    """Messages cut short: by whole 16-byte blocks (the size no longer matches
    the offset table: both reject); cut with the offset table's last entry
    set to the shorter data region (the last chunk loses its tail: the
    verdicts agree); cut to a size that is not a multiple of 16 bytes, or
    into the header (an argument error before anything runs)."""
    rng = np.random.default_rng(zlib.crc32(repr(("trunc", kind)).encode()))
    m, ref, gpu, torch = message(rlib, orc, kind, rng)
    n_chunks = -(-N_SYM // CS)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    for cut in (16, 48, 160):
        bad = m[:m.size - cut].copy()
        with pytest.raises(oracle.OracleError):
            ref(bad)
        assert _gpu_status(torch, gpu, bad, cuda)[1] == rlib.RANS_ERR_CORRUPT, cut
        fixed = bad.copy()
        offs = fixed[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
        offs[n_chunks] = np.uint32(fixed.size - data0)
        try:
            want = ref(fixed)
        except oracle.OracleError:
            want = None
        out, st = _gpu_status(torch, gpu, fixed, cuda)
        if want is None:
            assert st == rlib.RANS_ERR_CORRUPT, cut
        else:
            assert st == rlib.RANS_OK and np.array_equal(out.cpu().numpy(), want), cut
    for size in (m.size - 1, m.size - 7, data0 - 16, 16):
        with pytest.raises(rlib.RansError) as e:
            gpu(torch.from_numpy(m[:size].copy()).to(cuda))
        assert e.value.code == rlib.RANS_ERR_INVALID_ARG, size
