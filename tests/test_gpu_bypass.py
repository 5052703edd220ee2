"""Bypass (raw words interleaved with the coded symbols, Section 3) on the
GPU against the CPU oracle: encoded messages byte for byte, decoded symbols
and raw words exactly; edge sizes; version mismatch in both directions."""
import itertools
import zlib

import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def model(rlib, kind, rng):
    if kind == "zipf256":
        p = wl.zipf_probs(256, 1.1)
    elif kind == "dirichlet":
        p = wl.dirichlet_probs(rng, int(rng.integers(16, 257)), 0.3)
    elif kind == "binary":
        p0 = float(rng.uniform(0.5, 0.999))
        p = np.array([p0, 1 - p0])
    elif kind == "single":
        p = np.array([1.0])
    else:
        raise ValueError(kind)
    return rlib.rans_quantize_table(wl.weights_from_probs(p))


def flags_for(pattern, n_alpha, rng):
    if pattern == "none":
        return np.zeros(n_alpha, np.uint8)
    if pattern == "all":
        return np.ones(n_alpha, np.uint8)
    return (rng.random(n_alpha) < 0.4).astype(np.uint8)


def draw(rng, freq, n):
    return rng.choice(len(freq), size=n, p=freq / freq.sum()).astype(np.uint8)


def gpu_pair(rlib, cuda, sym, raw, freq, flags, N, CS):
    import torch

    d_sym = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                          device=cuda)
    d_raw = (torch.from_numpy(raw.view(np.int16)).to(cuda) if raw.size
             else torch.empty(0, dtype=torch.int16, device=cuda))
    msg, _, _ = rlib.encode_bypass(d_sym, d_raw, freq, flags, N, CS)
    out, rout, _ = rlib.decode_bypass(msg, sym.size, freq, flags, N, CS)
    return (msg.cpu().numpy(), out.cpu().numpy(), rout.cpu().numpy().view(np.uint16))


CASES = list(itertools.product(["zipf256", "dirichlet", "binary", "single"],
                               ["none", "all", "some"], [32, 7, 1], [4096, 1000]))


@pytest.mark.parametrize("kind,pattern,N,CS", CASES)
def test_bypass_matches_oracle(rlib, orc, cuda, kind, pattern, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr((kind, pattern, N, CS)).encode()))
    freq = model(rlib, kind, rng)
    flags = flags_for(pattern, len(freq), rng)
    n = 3 * CS + CS // 3 + 5
    sym = draw(rng, freq, n)
    raw = rng.integers(0, 1 << 16, size=n).astype(np.uint16)
    msg, out, rout = gpu_pair(rlib, cuda, sym, raw, freq, flags, N, CS)
    ref = orc.encode_message_bypass(sym, raw, freq, flags, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    want_raw = np.where(flags[sym] == 1, raw, 0).astype(np.uint16)
    assert np.array_equal(out, sym)
    assert np.array_equal(rout, want_raw)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 65, 4097])
def test_bypass_edge_sizes(rlib, orc, cuda, n):
    rng = np.random.default_rng(n + 5)
    freq = model(rlib, "dirichlet", rng)
    flags = flags_for("some", len(freq), rng)
    flags[0] = 1
    sym = draw(rng, freq, n)
    raw = rng.integers(0, 1 << 16, size=n).astype(np.uint16)
    for N, CS in ((32, 64), (5, 33)):
        msg, out, rout = gpu_pair(rlib, cuda, sym, raw, freq, flags, N, CS)
        assert np.array_equal(msg, orc.encode_message_bypass(sym, raw, freq, flags, N=N,
                                                              chunk_symbols=CS))
        assert np.array_equal(out, sym)
        assert np.array_equal(rout, np.where(flags[sym] == 1, raw, 0).astype(np.uint16))


def test_bypass_decodes_oracle_messages_and_checks_version(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(77)
    freq = model(rlib, "zipf256", rng)
    flags = flags_for("some", 256, rng)
    n = 200_003
    sym = draw(rng, freq, n)
    raw = rng.integers(0, 1 << 16, size=n).astype(np.uint16)
    ref = orc.encode_message_bypass(sym, raw, freq, flags, N=32, chunk_symbols=16384)
    d_ref = torch.from_numpy(ref).to(cuda)
    out, rout, _ = rlib.decode_bypass(d_ref, n, freq, flags, 32, 16384)
    assert np.array_equal(out.cpu().numpy(), sym)
    assert np.array_equal(rout.cpu().numpy().view(np.uint16), np.where(flags[sym] == 1, raw, 0))
    # the plain decoder refuses a bypass message, and the reverse
    _, st = rlib.decode(d_ref, n, freq, 32, 16384, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    plain = torch.from_numpy(orc.encode_message(sym, freq, N=32, chunk_symbols=16384)).to(cuda)
    _, _, st = rlib.decode_bypass(plain, n, freq, flags, 32, 16384, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    # a flipped raw flag in the model is damage the decoder notices
    wrong = flags.copy()
    wrong[int(sym[0])] ^= 1
    _, _, st = rlib.decode_bypass(d_ref, n, freq, wrong, 32, 16384, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT


def test_bypass_many_chunks(rlib, orc, cuda):
    """Several waves of chunks; sampled chunks checked against the oracle."""
    import torch

    rng = np.random.default_rng(91)
    freq = model(rlib, "zipf256", rng)
    flags = (np.arange(256) >= 16).astype(np.uint8)       # rarer symbols carry a word
    CS, n_chunks = 4096, 20_000
    n = CS * n_chunks - 777
    sym = draw(rng, freq, n)
    raw = rng.integers(0, 1 << 16, size=n).astype(np.uint16)
    msg, out, rout = gpu_pair(rlib, cuda, sym, raw, freq, flags, 32, CS)
    assert np.array_equal(out, sym)
    assert np.array_equal(rout, np.where(flags[sym] == 1, raw, 0))
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = msg[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)
    for c in rng.choice(n_chunks, size=12, replace=False):
        c = int(c)
        a, z = c * CS, min(n, (c + 1) * CS)
        ref = orc.encode_chunk_bypass(sym[a:z], raw[a:z], freq, flags, N=32)
        assert np.array_equal(msg[data0 + offs[c]:data0 + offs[c + 1]], ref), c
