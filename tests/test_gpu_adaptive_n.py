"""Adaptive models over n <= 16 symbols, one per coder (Section 5: adaptive
models vectorize while every lane updates only its own model), on the GPU
against the CPU oracle: every message byte for byte, every decode symbol for
symbol (zero tolerance), at every register size of the model (n up to 4, 8,
16), with partial steps and ragged chunks; symbols outside the alphabet and a
wrong alphabet size are reported, not decoded."""
import zlib

import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [(n, N, CS) for n in (2, 3, 4, 5, 8, 9, 16) for N, CS in ((32, 4096), (7, 1000), (1, 333))]


@pytest.mark.parametrize("n,N,CS", CASES)
def test_adaptive_n_matches_oracle(rlib, orc, cuda, n, N, CS):
    import torch

    rng = np.random.default_rng(zlib.crc32(repr(("adaptn", n, N, CS)).encode()))
    sym = wl.drifting_symbols(rng, 3 * CS + CS // 3 + 5, n, 700, 0.4)
    d = torch.from_numpy(sym).to(cuda)
    msg, _, _ = rlib.encode_adaptive_n(d, n, N, CS)
    ref = orc.encode_message_adaptive_n(sym, n, N=N, chunk_symbols=CS)
    assert np.array_equal(msg.cpu().numpy(), ref)
    out, _ = rlib.decode_adaptive_n(torch.from_numpy(ref).to(cuda), sym.size, n, N, CS)
    assert np.array_equal(out.cpu().numpy(), sym)


@pytest.mark.parametrize("n_sym", [0, 1, 31, 32, 33, 65, 4097])
def test_adaptive_n_edge_sizes(rlib, orc, cuda, n_sym):
    import torch

    rng = np.random.default_rng(n_sym + 5)
    sym = rng.integers(0, 6, size=n_sym).astype(np.uint8)
    d = torch.from_numpy(sym).to(cuda) if n_sym else torch.empty(0, dtype=torch.uint8, device=cuda)
    msg, _, _ = rlib.encode_adaptive_n(d, 6, 32, 64)
    assert np.array_equal(msg.cpu().numpy(), orc.encode_message_adaptive_n(sym, 6, N=32,
                                                                           chunk_symbols=64))
    out, _ = rlib.decode_adaptive_n(msg, n_sym, 6, 32, 64)
    assert np.array_equal(out.cpu().numpy(), sym)


def test_adaptive_n_long_chunk(rlib, orc, cuda):
    """One chunk of 200,003 symbols over 16 (hundreds of ring segments), a
    source the models must keep re-learning."""
    import torch

    rng = np.random.default_rng(61)
    sym = wl.drifting_symbols(rng, 200_003, 16, 4096, 0.3)
    d = torch.from_numpy(sym).to(cuda)
    msg, _, _ = rlib.encode_adaptive_n(d, 16, 32, 1 << 20)
    assert np.array_equal(msg.cpu().numpy(),
                          orc.encode_message_adaptive_n(sym, 16, N=32, chunk_symbols=1 << 20))
    out, _ = rlib.decode_adaptive_n(msg, sym.size, 16, 32, 1 << 20)
    assert torch.equal(out, d)


def test_adaptive_n_bad_symbol_and_wrong_alphabet(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(67)
    sym = rng.integers(0, 5, size=20_000).astype(np.uint8)
    bad = sym.copy()
    bad[12_345] = 5                       # outside an alphabet of 5
    with pytest.raises(rlib.RansError) as e:
        rlib.encode_adaptive_n(torch.from_numpy(bad).to(cuda), 5, 32, 4096)
    assert e.value.code == rlib.RANS_ERR_ZERO_FREQ
    msg, _, _ = rlib.encode_adaptive_n(torch.from_numpy(sym).to(cuda), 5, 32, 4096)
    with pytest.raises(rlib.RansError) as e:   # the header records n = 5
        rlib.decode_adaptive_n(msg, sym.size, 6, 32, 4096)
    assert e.value.code == rlib.RANS_ERR_CORRUPT
    for n_bad in (0, 1, 17):
        out = torch.empty(16, dtype=torch.uint8, device=cuda)
        st = torch.zeros(1, dtype=torch.int32, device=cuda)
        assert rlib.rans_decode_adaptive_n(msg, msg.numel(), n_bad, 32, 4096, out, 16, st,
                                           check=False) == rlib.RANS_ERR_INVALID_ARG


def test_adaptive_n_full_size_sampled(rlib, orc, cuda):
    """The benchmark's workload (256 Mi symbols over 16, Dirichlet(0.5) runs
    of 4096, 4096 chunks of 64 Ki, N = 32): round trip on the device, and
    sampled chunks re-encoded and decoded by the oracle one by one."""
    import torch

    cfg = wl.WORKLOADS["adaptive_n"]
    n, k, N, CS = cfg["n_symbols"], cfg["n_alpha"], cfg["n_lanes"], cfg["chunk_symbols"]
    d = wl.drifting_symbols_device(n, k, cfg["segment"], wl.seed_for("adaptive_n"), cuda,
                                   cfg["dirichlet"])
    msg, _, _ = rlib.encode_adaptive_n(d, k, N, CS)
    out, _ = rlib.decode_adaptive_n(msg, n, k, N, CS)
    assert torch.equal(out, d)
    n_chunks = n // CS
    offs = msg[32:32 + 4 * (n_chunks + 1)].cpu().numpy().view(np.uint32).astype(np.int64)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    for c in (0, 1, 777, n_chunks - 1):
        chunk_sym = d[c * CS:(c + 1) * CS].cpu().numpy()
        gpu_chunk = msg[data0 + offs[c]:data0 + offs[c + 1]].cpu().numpy()
        assert np.array_equal(gpu_chunk, orc.encode_chunk_adaptive_n(chunk_sym, k, N=N)), c
        assert np.array_equal(orc.decode_chunk_adaptive_n(gpu_chunk, CS, k, N=N), chunk_sym), c
