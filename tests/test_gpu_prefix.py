"""Prefix-code coders interleaved by their decoders' read order (Section 4:
the encoder runs the decoder's reads and lays the words down where they
will be read) on the GPU against the CPU oracle's instrumented-decoder mux,
byte for byte."""
import itertools
import zlib

import numpy as np
import pytest

import oracle
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def code(orc, kind, rng):
    """(lengths, symbol probabilities) of a test code."""
    if kind == "zipf256":
        p = wl.zipf_probs(256, 1.1)
    elif kind == "dirichlet":
        p = wl.dirichlet_probs(rng, int(rng.integers(16, 257)), 0.3)
    elif kind == "binary":
        p = np.array([0.9, 0.1])
    elif kind == "uniform256":
        p = np.full(256, 1 / 256)
    elif kind == "single":              # one symbol: an incomplete code of one 1-bit word
        p = np.array([1.0])
    elif kind == "long":                # the 12-bit limit binds: many 12-bit codes in use
        p = 0.5 ** np.arange(1, 41)
        p /= p.sum()
    else:
        raise ValueError(kind)
    ln = orc.prefix_lengths(wl.weights_from_probs(p), 12)
    return ln, p


def draw(rng, p, n, kind):
    if kind == "long":                  # mostly the rare, long codes
        return rng.integers(0, len(p), size=n).astype(np.uint8)
    return rng.choice(len(p), size=n, p=p).astype(np.uint8)


def gpu_pair(rlib, cuda, sym, ln, N, CS):
    import torch

    d = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                      device=cuda)
    msg, _, _ = rlib.encode_prefix(d, ln, N, CS)
    out, _ = rlib.decode_prefix(msg, sym.size, ln, N, CS)
    return msg.cpu().numpy(), out.cpu().numpy()


CASES = list(itertools.product(["zipf256", "dirichlet", "binary", "uniform256", "single", "long"],
                               [32, 7, 1], [4096, 1001]))


@pytest.mark.parametrize("kind,N,CS", CASES)
def test_prefix_match_oracle(rlib, orc, cuda, kind, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr(("prefix", kind, N, CS)).encode()))
    ln, p = code(orc, kind, rng)
    n = 3 * CS + CS // 3 + 5
    sym = draw(rng, p, n, kind)
    msg, out = gpu_pair(rlib, cuda, sym, ln, N, CS)
    ref = orc.encode_message_prefix(sym, ln, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(out, sym)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 4097])
def test_prefix_edge_sizes(rlib, orc, cuda, n):
    rng = np.random.default_rng(n + 17)
    ln, p = code(orc, "long", rng)
    sym = draw(rng, p, n, "long")
    for N, CS in ((32, 64), (5, 33), (1, 7), (32, 65536)):
        msg, out = gpu_pair(rlib, cuda, sym, ln, N, CS)
        assert np.array_equal(msg, orc.encode_message_prefix(sym, ln, N=N, chunk_symbols=CS))
        assert np.array_equal(out, sym)


def test_prefix_rejects_symbols_without_code(rlib, orc, cuda):
    import torch

    ln = np.array([1, 2, 0, 2], dtype=np.uint8)
    sym = np.zeros(5000, dtype=np.uint8)
    sym[3333] = 2
    _, _, st = rlib.encode_prefix(torch.from_numpy(sym).to(cuda), ln, 32, 1024, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_ZERO_FREQ
    sym[3333] = 9                                   # beyond the alphabet
    _, _, st = rlib.encode_prefix(torch.from_numpy(sym).to(cuda), ln, 32, 1024, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_ZERO_FREQ
    d = torch.zeros(16, dtype=torch.uint8, device=cuda)
    for bad in (np.array([1, 1, 1], dtype=np.uint8), np.array([13, 1], dtype=np.uint8),
                np.zeros(3, dtype=np.uint8)):
        with pytest.raises(rlib.RansError):
            rlib.encode_prefix(d, bad, 32, 1024)


def test_prefix_kind_is_checked(rlib, orc, cuda):
    """Prefix and plain decoders refuse each other's messages; a prefix
    message decodes only with its own N."""
    import torch

    rng = np.random.default_rng(71)
    ln, p = code(orc, "zipf256", rng)
    n = 20_000
    sym = draw(rng, p, n, "zipf256")
    m32, _ = gpu_pair(rlib, cuda, sym, ln, 32, 4096)
    m16, _ = gpu_pair(rlib, cuda, sym, ln, 16, 4096)
    assert m32.size != m16.size or not np.array_equal(m32, m16)
    d32 = torch.from_numpy(m32).to(cuda)
    _, st = rlib.decode_prefix(d32, n, ln, 16, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    _, st = rlib.decode(d32, n, freq, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    plain = torch.from_numpy(orc.encode_message(sym, freq, N=32, chunk_symbols=4096)).to(cuda)
    _, st = rlib.decode_prefix(plain, n, ln, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT


def test_prefix_decode_oracle_messages_and_damage(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(73)
    ln, p = code(orc, "dirichlet", rng)
    n = 300_007
    sym = draw(rng, p, n, "dirichlet")
    ref = orc.encode_message_prefix(sym, ln, N=32, chunk_symbols=8192)
    out, _ = rlib.decode_prefix(torch.from_numpy(ref).to(cuda), n, ln, 32, 8192)
    assert np.array_equal(out.cpu().numpy(), sym)
    n_chunks = -(-n // 8192)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = ref[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    for c, pos, bit in ((3, 500, 1), (7, 1000, 6), (20, 77, 0), (0, 3, 7), (36, 1, 3),
                        (11, 9000, 5)):
        bad = ref.copy()
        a, z = data0 + int(offs[c]), data0 + int(offs[c + 1])
        bad[a + pos % (z - a)] ^= 1 << bit
        try:
            want = orc.decode_message_prefix(bad, n, ln, N=32, chunk_symbols=8192)
        except oracle.OracleError:
            want = None
        out, st = rlib.decode_prefix(torch.from_numpy(bad).to(cuda), n, ln, 32, 8192, sync=False)
        torch.cuda.synchronize()
        if want is None:
            assert int(st.item()) == rlib.RANS_ERR_CORRUPT
        else:
            assert int(st.item()) == rlib.RANS_OK
            assert np.array_equal(out.cpu().numpy(), want)


def test_prefix_full_size_sampled_parity(rlib, orc, cuda):
    """The 1 GiB Zipf(1.1) workload as a prefix-code message (16384 chunks
    of 64 Ki, 32 coders) in the launch configuration the benchmark times:
    full round trip on the device, sampled chunks re-encoded and decoded by
    the oracle one by one."""
    import torch

    cfg = wl.WORKLOADS["chunked"]
    n, N, CS = cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    ln = orc.prefix_lengths(wl.weights_from_probs(p), 12)
    d = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), cuda)
    msg, _, _ = rlib.encode_prefix(d, ln, N, CS)
    out, _ = rlib.decode_prefix(msg, n, ln, N, CS)
    assert torch.equal(out, d)
    n_chunks = n // CS
    head = msg[: 32 + 4 * (n_chunks + 1)].cpu().numpy()
    h = head[:32].view(np.uint32)
    assert list(h[:4]) == [0x534E4152, 5, N, 12] and list(h[6:8]) == [CS, n_chunks]
    offs = head[32:].view(np.uint32).astype(np.int64)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    rng = np.random.default_rng(79)
    picks = sorted({0, n_chunks - 1, *rng.integers(0, n_chunks, size=5).tolist()})
    for c in picks:
        chunk_sym = d[c * CS:(c + 1) * CS].cpu().numpy()
        gpu_chunk = msg[data0 + offs[c]: data0 + offs[c + 1]].cpu().numpy()
        assert np.array_equal(gpu_chunk, orc.encode_chunk_prefix(chunk_sym, ln, N=N)), c
        assert np.array_equal(orc.decode_chunk_prefix(gpu_chunk, CS, ln, N=N), chunk_sym), c
