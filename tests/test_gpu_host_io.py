"""rans_decode_host and rans_encode_host: decoding and encoding from and to
host memory with the copies overlapped with the coding, against the CPU
oracle byte for byte.  Sizes span several pieces (a piece is about 32 Mi
symbols of whole chunks)."""
import numpy as np
import pytest

import oracle
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def pinned(a):
    import torch

    t = torch.empty(a.size, dtype=torch.uint8, pin_memory=True)
    t.numpy()[:] = a
    return t


@pytest.fixture(scope="module")
def big(rlib, orc):
    rng = np.random.default_rng(2024)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
    n = 3 * (32 << 20) + 12345              # three full pieces and a ragged fourth
    sym = wl.iid_symbols(rng, freq / freq.sum(), n)
    msg = orc.encode_message(sym, freq, N=32, chunk_symbols=65536)
    return freq, sym, msg


def test_host_decode_matches_oracle(rlib, cuda, big):
    freq, sym, msg = big
    out, st = rlib.decode_host(pinned(msg), sym.size, freq, 32, 65536, device=cuda)
    assert st == rlib.RANS_OK
    assert np.array_equal(out.numpy(), sym)


def test_host_decode_damage_like_the_oracle(rlib, orc, cuda, big):
    """One flipped bit in a word of the third piece.  rANS carries no
    redundancy but the final states, so some flips decode to other symbols
    with every check passing: then the GPU must produce exactly the oracle's
    symbols; a flip the oracle rejects must give RANS_ERR_CORRUPT."""
    freq, sym, msg = big
    n_chunks = -(-sym.size // 65536)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = msg[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    c = 2 * 512 + 7
    a, z = data0 + int(offs[c]), data0 + int(offs[c + 1])
    seen = set()
    for pos, bit in ((100, 2), (101, 7), (2000, 0), (30000, 5)):
        bad = msg.copy()
        bad[a + 4 * 32 + pos] ^= 1 << bit
        try:
            ref = orc.decode_chunk(bad[a:z], 65536, freq, N=32)
        except oracle.OracleError:
            ref = None
        out, st = rlib.decode_host(pinned(bad), sym.size, freq, 32, 65536, device=cuda)
        if ref is None:
            assert st == rlib.RANS_ERR_CORRUPT, (pos, bit)
        else:
            assert st == rlib.RANS_OK, (pos, bit)
            got = out.numpy()
            assert np.array_equal(got[c * 65536:(c + 1) * 65536], ref), (pos, bit)
            assert np.array_equal(np.delete(got, np.s_[c * 65536:(c + 1) * 65536]),
                                  np.delete(sym, np.s_[c * 65536:(c + 1) * 65536]))
        seen.add(ref is None)
    assert True in seen                     # at least one detected flip
    bad = msg.copy()                        # offsets not increasing: one piece, reported
    bad[32 + 4 * 600:32 + 4 * 601] = np.frombuffer(np.uint32(0xFFFFFF00).tobytes(), np.uint8)
    _, st = rlib.decode_host(pinned(bad), sym.size, freq, 32, 65536, device=cuda)
    assert st == rlib.RANS_ERR_CORRUPT


def test_host_decode_small_and_pageable(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(7)
    for n, N, CS in ((0, 32, 4096), (1, 32, 4096), (100_003, 7, 1000), (2_000_000, 32, 65536)):
        freq = rlib.rans_quantize_table(wl.weights_from_probs(wl.dirichlet_probs(rng, 100, 0.3)))
        sym = wl.iid_symbols(rng, freq / freq.sum(), n)
        msg = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
        h_msg = torch.from_numpy(msg.copy())          # pageable
        out = torch.zeros(max(1, n), dtype=torch.uint8)
        work = torch.empty(rlib.rans_decode_host_work_size(msg.size, n), dtype=torch.uint8,
                           device=cuda)
        status = torch.full((1,), 99, dtype=torch.int32)
        rlib.rans_decode_host(h_msg, msg.size, freq, N, CS, out, n, status, work, work.numel())
        torch.cuda.synchronize()
        assert int(status.item()) == rlib.RANS_OK
        assert np.array_equal(out.numpy()[:n], sym)
    with pytest.raises(rlib.RansError) as e:
        rlib.rans_decode_host(h_msg, msg.size, freq, 32, 65536, out, n, status, work, 16)
    assert e.value.code == rlib.RANS_ERR_BUFFER_TOO_SMALL


# ---------------------------------------------------------------------------
# rans_encode_host: symbols and message in host memory
# ---------------------------------------------------------------------------

def test_host_encode_matches_oracle(rlib, cuda, big):
    """Page-locked input and output: the device writes the message straight
    into host memory piece by piece (four pieces here)."""
    freq, sym, msg = big
    out, st = rlib.encode_host(pinned(sym), freq, 32, 65536, device=cuda)
    assert st == rlib.RANS_OK
    assert np.array_equal(out.numpy(), msg)


def test_host_encode_pageable_and_misaligned_outputs(rlib, cuda, big):
    """A pageable output (and pageable input), and a page-locked output that
    is not 16-byte aligned, take the staged path: same message."""
    import torch

    freq, sym, msg = big
    n = 40 << 20                                      # two pieces
    cap = rlib.rans_max_encoded_size(n, 32, 65536)
    pageable = torch.empty(cap, dtype=torch.uint8)
    got, st = rlib.encode_host(torch.from_numpy(sym[:n].copy()), freq, 32, 65536, device=cuda,
                               out=pageable)
    assert st == rlib.RANS_OK
    ref_msg = oracle.default().encode_message(sym[:n], freq, N=32, chunk_symbols=65536)
    assert np.array_equal(got.numpy(), ref_msg)
    base = torch.empty(cap + 16, dtype=torch.uint8, pin_memory=True)
    shifted = base[4:4 + cap]
    got, st = rlib.encode_host(pinned(sym[:n]), freq, 32, 65536, device=cuda, out=shifted)
    assert st == rlib.RANS_OK
    assert np.array_equal(got.numpy(), ref_msg)


@pytest.mark.parametrize("n,N,CS", [(0, 32, 65536), (1, 32, 65536), (33, 7, 4), (100_003, 5, 999)])
def test_host_encode_small(rlib, orc, cuda, n, N, CS):
    rng = np.random.default_rng(n + N)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(40, 1.0)))
    sym = wl.iid_symbols(rng, freq / freq.sum(), n)
    out, st = rlib.encode_host(pinned(sym), freq, N, CS, device=cuda)
    assert st == rlib.RANS_OK
    assert np.array_equal(out.numpy(), orc.encode_message(sym, freq, N=N, chunk_symbols=CS))


def test_host_encode_zero_frequency_symbol(rlib, cuda):
    freq = np.zeros(4, dtype=np.uint16)
    freq[:3] = [2048, 1024, 1024]
    sym = np.zeros(300_000, dtype=np.uint8)
    sym[123_456] = 3
    out, st = rlib.encode_host(pinned(sym), freq, 32, 4096, device=cuda)
    assert st == rlib.RANS_ERR_ZERO_FREQ
    assert out.numel() == 0
