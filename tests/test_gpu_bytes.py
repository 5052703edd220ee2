"""Byte-wise messages (b = 2^8 < M, two renormalization digits per symbol at
most, read breadth-first across the N lanes of a step -- Section 5) on the
GPU against the CPU oracle, byte for byte."""
import itertools
import zlib

import numpy as np
import pytest

import oracle
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
    elif kind == "uniform256":
        p = np.full(256, 1 / 256)
    elif kind == "single":
        p = np.array([1.0])
    elif kind == "rare":              # many f = 1 symbols drawn often: two digits per symbol
        p = np.full(200, 1.0)
        p[0] = 1e6
        p /= p.sum()
    else:
        raise ValueError(kind)
    return rlib.rans_quantize_table(wl.weights_from_probs(p))


def draw(rng, freq, n, kind):
    if kind == "rare":
        return rng.integers(0, len(freq), size=n).astype(np.uint8)
    return rng.choice(len(freq), size=n, p=freq / freq.sum()).astype(np.uint8)


def gpu_pair(rlib, cuda, sym, freq, N, CS):
    import torch

    d = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                      device=cuda)
    msg, _, _ = rlib.encode_bytes(d, freq, N, CS)
    out, _ = rlib.decode_bytes(msg, sym.size, freq, N, CS)
    return msg.cpu().numpy(), out.cpu().numpy()


CASES = list(itertools.product(["zipf256", "dirichlet", "binary", "uniform256", "single", "rare"],
                               [32, 7, 1], [4096, 1001]))


@pytest.mark.parametrize("kind,N,CS", CASES)
def test_bytes_match_oracle(rlib, orc, cuda, kind, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr(("bytes", kind, N, CS)).encode()))
    freq = model(rlib, kind, rng)
    n = 3 * CS + CS // 3 + 5
    sym = draw(rng, freq, n, kind)
    msg, out = gpu_pair(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message_bytes(sym, freq, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(out, sym)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 4097])
def test_bytes_edge_sizes(rlib, orc, cuda, n):
    rng = np.random.default_rng(n + 9)
    freq = model(rlib, "rare", rng)
    sym = draw(rng, freq, n, "rare")
    for N, CS in ((32, 64), (5, 33), (1, 7)):
        msg, out = gpu_pair(rlib, cuda, sym, freq, N, CS)
        assert np.array_equal(msg, orc.encode_message_bytes(sym, freq, N=N, chunk_symbols=CS))
        assert np.array_equal(out, sym)


def test_width_is_baked_in(rlib, orc, cuda):
    """The same symbols give different streams at different N (the digits of
    a step are read breadth-first across its lanes), each decodes only with
    its own N, and the plain and byte-wise decoders refuse each other's
    messages."""
    import torch

    rng = np.random.default_rng(31)
    freq = model(rlib, "rare", rng)
    n = 20_000
    sym = draw(rng, freq, n, "rare")
    m32, _ = gpu_pair(rlib, cuda, sym, freq, 32, 4096)
    m16, _ = gpu_pair(rlib, cuda, sym, freq, 16, 4096)
    assert m32.size != m16.size or not np.array_equal(m32, m16)
    d32 = torch.from_numpy(m32).to(cuda)
    _, st = rlib.decode_bytes(d32, n, freq, 16, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    _, st = rlib.decode(d32, n, freq, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    plain = torch.from_numpy(orc.encode_message(sym, freq, N=32, chunk_symbols=4096)).to(cuda)
    _, st = rlib.decode_bytes(plain, n, freq, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT


def test_bytes_decode_oracle_messages_and_damage(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(37)
    freq = model(rlib, "zipf256", rng)
    n = 300_007
    sym = draw(rng, freq, n, "zipf256")
    ref = orc.encode_message_bytes(sym, freq, N=32, chunk_symbols=8192)
    out, _ = rlib.decode_bytes(torch.from_numpy(ref).to(cuda), n, freq, 32, 8192)
    assert np.array_equal(out.cpu().numpy(), sym)
    n_chunks = -(-n // 8192)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = ref[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    for c, pos, bit in ((3, 500, 1), (7, 2000, 6), (20, 77, 0)):
        bad = ref.copy()
        a, z = data0 + int(offs[c]), data0 + int(offs[c + 1])
        bad[a + 4 * 32 + pos] ^= 1 << bit
        try:
            want = orc.decode_chunk_bytes(bad[a:z], 8192, freq, N=32)
        except oracle.OracleError:
            want = None
        out, st = rlib.decode_bytes(torch.from_numpy(bad).to(cuda), n, freq, 32, 8192,
                                    sync=False)
        torch.cuda.synchronize()
        if want is None:
            assert int(st.item()) == rlib.RANS_ERR_CORRUPT
        else:
            assert int(st.item()) == rlib.RANS_OK
            assert np.array_equal(out.cpu().numpy()[c * 8192:(c + 1) * 8192], want)


# Chunk counts on both sides of the decoder's switch on a B300 (148 SMs):
# messages of up to 3552 chunks take the latency form (both digit passes
# issued together, chunks dealt warp-major), larger ones the two-pass form.
@pytest.mark.parametrize("n_chunks,N,kind", [(1, 32, "rare"), (148, 32, "rare"), (3552, 32, "rare"),
                                             (3553, 32, "rare"), (4736, 32, "rare"),
                                             (3552, 32, "zipf256"), (3553, 32, "zipf256"),
                                             (3552, 7, "rare"), (3553, 7, "rare")])
def test_bytes_every_launch_shape(rlib, orc, cuda, n_chunks, N, kind):
    """A byte-wise message of n_chunks chunks of 96 symbols (the last one
    ragged) is the oracle's, and the oracle's message decodes back, whichever
    form of the step the decoder launches for it."""
    import torch

    CS = 96
    rng = np.random.default_rng(n_chunks * 100 + N + len(kind))
    freq = model(rlib, kind, rng)
    sym = draw(rng, freq, (n_chunks - 1) * CS + 37, kind)
    msg, out = gpu_pair(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message_bytes(sym, freq, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(out, sym)
    back, _ = rlib.decode_bytes(torch.from_numpy(ref).to(cuda), sym.size, freq, N, CS)
    assert np.array_equal(back.cpu().numpy(), sym)


def test_bytes_many_chunks(rlib, orc, cuda):
    rng = np.random.default_rng(41)
    freq = model(rlib, "dirichlet", rng)
    CS, n_chunks = 4096, 12_000
    n = CS * n_chunks - 99
    sym = draw(rng, freq, n, "dirichlet")
    msg, out = gpu_pair(rlib, cuda, sym, freq, 32, CS)
    assert np.array_equal(out, sym)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = msg[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)
    for c in rng.choice(n_chunks, size=10, replace=False):
        c = int(c)
        ref = orc.encode_chunk_bytes(sym[c * CS:min(n, (c + 1) * CS)], freq, N=32)
        assert np.array_equal(msg[data0 + offs[c]:data0 + offs[c + 1]], ref), c
