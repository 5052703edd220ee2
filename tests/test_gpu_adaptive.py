"""Adaptive binary messages (one context per coder, so that no two lanes ever
update the same model -- Section 5) on the GPU against the CPU oracle, byte
for byte."""
import itertools
import zlib

import numpy as np
import pytest

import oracle
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def bits(rng, n, kind):
    if kind == "drifting":
        return wl.drifting_bits(rng, n, 4096)
    if kind == "short_drift":   # segments shorter than a context can follow
        return wl.drifting_bits(rng, n, 37)
    if kind == "zeros":         # contexts saturate at f_1 = 31
        return np.zeros(n, dtype=np.uint8)
    if kind == "ones":
        return np.ones(n, dtype=np.uint8)
    if kind == "alternating":   # each coder sees a constant bit iff N is even
        return (np.arange(n) & 1).astype(np.uint8)
    if kind == "half":
        return rng.integers(0, 2, size=n).astype(np.uint8)
    raise ValueError(kind)


def gpu_pair(rlib, cuda, sym, N, CS):
    import torch

    d = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                      device=cuda)
    msg, _, _ = rlib.encode_adaptive(d, N, CS)
    out, _ = rlib.decode_adaptive(msg, sym.size, N, CS)
    return msg.cpu().numpy(), out.cpu().numpy()


CASES = list(itertools.product(["drifting", "short_drift", "zeros", "ones", "alternating",
                                "half"], [32, 7, 1], [4096, 1001]))


@pytest.mark.parametrize("kind,N,CS", CASES)
def test_adaptive_match_oracle(rlib, orc, cuda, kind, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr(("adaptive", kind, N, CS)).encode()))
    n = 3 * CS + CS // 3 + 5
    sym = bits(rng, n, kind)
    msg, out = gpu_pair(rlib, cuda, sym, N, CS)
    ref = orc.encode_message_adaptive(sym, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(out, sym)
    assert np.array_equal(orc.decode_message_adaptive(msg, n, N=N, chunk_symbols=CS), sym)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 4097])
def test_adaptive_edge_sizes(rlib, orc, cuda, n):
    rng = np.random.default_rng(n + 13)
    sym = bits(rng, n, "drifting")
    for N, CS in ((32, 64), (5, 33), (1, 7), (32, 65536)):
        msg, out = gpu_pair(rlib, cuda, sym, N, CS)
        assert np.array_equal(msg, orc.encode_message_adaptive(sym, N=N, chunk_symbols=CS))
        assert np.array_equal(out, sym)


def test_adaptive_rejects_non_binary(rlib, cuda):
    """A symbol other than 0 or 1 has no frequency in a binary context."""
    import torch

    sym = np.zeros(5000, dtype=np.uint8)
    sym[4321] = 2
    d = torch.from_numpy(sym).to(cuda)
    _, _, st = rlib.encode_adaptive(d, 32, 1024, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_ZERO_FREQ


def test_adaptive_kind_is_checked(rlib, orc, cuda):
    """The plain and adaptive decoders refuse each other's messages, and an
    adaptive message decodes only with its own N."""
    import torch

    rng = np.random.default_rng(43)
    n = 20_000
    sym = bits(rng, n, "drifting")
    m32, _ = gpu_pair(rlib, cuda, sym, 32, 4096)
    m16, _ = gpu_pair(rlib, cuda, sym, 16, 4096)
    assert m32.size != m16.size or not np.array_equal(m32, m16)
    d32 = torch.from_numpy(m32).to(cuda)
    _, st = rlib.decode_adaptive(d32, n, 16, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    freq = np.array([2048, 2048], dtype=np.uint16)
    _, st = rlib.decode(d32, n, freq, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    plain = torch.from_numpy(orc.encode_message(sym, freq, N=32, chunk_symbols=4096)).to(cuda)
    _, st = rlib.decode_adaptive(plain, n, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT


def test_adaptive_beats_static_on_drifting_bits(rlib, orc, cuda):
    """On bits whose statistics drift, per-coder contexts code below the best
    single static binary model for the whole message."""
    import torch

    rng = np.random.default_rng(47)
    n = 1 << 20
    sym = bits(rng, n, "drifting")
    msg, out = gpu_pair(rlib, cuda, sym, 32, 65536)
    assert np.array_equal(out, sym)
    p1 = float(sym.mean())
    freq = rlib.rans_quantize_table(wl.weights_from_probs(np.array([1 - p1, p1])))
    static, _, _ = rlib.encode(torch.from_numpy(sym).to(cuda), freq, 32, 65536)
    assert msg.size < 0.85 * static.numel()   # 0.80 for this seed


def test_adaptive_decode_oracle_messages_and_damage(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(53)
    n = 300_007
    sym = bits(rng, n, "drifting")
    ref = orc.encode_message_adaptive(sym, N=32, chunk_symbols=8192)
    out, _ = rlib.decode_adaptive(torch.from_numpy(ref).to(cuda), n, 32, 8192)
    assert np.array_equal(out.cpu().numpy(), sym)
    n_chunks = -(-n // 8192)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = ref[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    for c, pos, bit in ((3, 500, 1), (7, 1000, 6), (20, 77, 0), (0, 3, 7), (9, 0, 0)):
        bad = ref.copy()
        a, z = data0 + int(offs[c]), data0 + int(offs[c + 1])
        bad[a + 4 * 32 + pos % (z - a - 4 * 32)] ^= 1 << bit   # a word of chunk c
        try:
            want = orc.decode_message_adaptive(bad, n, N=32, chunk_symbols=8192)
        except oracle.OracleError:
            want = None
        out, st = rlib.decode_adaptive(torch.from_numpy(bad).to(cuda), n, 32, 8192, sync=False)
        torch.cuda.synchronize()
        if want is None:
            assert int(st.item()) == rlib.RANS_ERR_CORRUPT
        else:
            assert int(st.item()) == rlib.RANS_OK
            assert np.array_equal(out.cpu().numpy(), want)


def test_adaptive_full_size_sampled_parity(rlib, orc, cuda):
    """The 256 Mi-bit adaptive workload (4096 chunks of 64 Ki, 32 coders) in
    the launch configuration the benchmark times: full round trip on the
    device, sampled chunks re-encoded and decoded by the oracle one by one."""
    import torch

    cfg = wl.WORKLOADS["adaptive"]
    n, N, CS = cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    d = wl.drifting_bits_device(n, cfg["segment"], wl.seed_for("adaptive"), cuda,
                                cfg["p0_lo"], cfg["p0_hi"])
    msg, _, _ = rlib.encode_adaptive(d, N, CS)
    out, _ = rlib.decode_adaptive(msg, n, N, CS)
    assert torch.equal(out, d)
    n_chunks = n // CS
    head = msg[: 32 + 4 * (n_chunks + 1)].cpu().numpy()
    h = head[:32].view(np.uint32)
    assert list(h[:4]) == [0x534E4152, 4, N, 12] and list(h[6:8]) == [CS, n_chunks]
    offs = head[32:].view(np.uint32).astype(np.int64)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    rng = np.random.default_rng(61)
    picks = sorted({0, n_chunks - 1, *rng.integers(0, n_chunks, size=5).tolist()})
    for c in picks:
        chunk_sym = d[c * CS:(c + 1) * CS].cpu().numpy()
        gpu_chunk = msg[data0 + offs[c]: data0 + offs[c + 1]].cpu().numpy()
        assert np.array_equal(gpu_chunk, orc.encode_chunk_adaptive(chunk_sym, N=N)), c
        assert np.array_equal(orc.decode_chunk_adaptive(gpu_chunk, CS, N=N), chunk_sym), c
