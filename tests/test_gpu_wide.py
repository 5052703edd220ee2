"""Plain messages at 13 and 14 bits of probability resolution (M = 2^13 or
2^14 with b = 2^16: still one renormalization per symbol, Section 5) on the
GPU against the CPU oracle, byte for byte.  The model's sum selects M; the
header records log2 M."""
import itertools
import zlib

import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def model(rlib, kind, lm, rng):
    if kind == "zipf256":
        p = wl.zipf_probs(256, 1.1)
    elif kind == "dirichlet":
        p = wl.dirichlet_probs(rng, int(rng.integers(16, 257)), 0.3)
    elif kind == "binary":
        p = np.array([0.999, 0.001])
    elif kind == "single":
        p = np.array([1.0])
    elif kind == "rare":                 # many symbols at the smallest frequency
        p = np.full(256, 1.0)
        p[0] = 1e7
        p /= p.sum()
    else:
        raise ValueError(kind)
    return rlib.rans_quantize_table(wl.weights_from_probs(p), lm), p


def draw(rng, p, n, kind):
    if kind == "rare":
        return rng.integers(0, len(p), size=n).astype(np.uint8)
    return rng.choice(len(p), size=n, p=p).astype(np.uint8)


def gpu_pair(rlib, cuda, sym, freq, N, CS):
    import torch

    d = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                      device=cuda)
    msg, _, _ = rlib.encode(d, freq, N, CS)
    out, _ = rlib.decode(msg, sym.size, freq, N, CS)
    return msg.cpu().numpy(), out.cpu().numpy()


CASES = list(itertools.product([13, 14], ["zipf256", "dirichlet", "binary", "single", "rare"],
                               [32, 7, 1], [4096, 1001]))


@pytest.mark.parametrize("lm,kind,N,CS", CASES)
def test_wide_match_oracle(rlib, orc, cuda, lm, kind, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr(("wide", lm, kind, N, CS)).encode()))
    freq, p = model(rlib, kind, lm, rng)
    assert int(freq.astype(np.int64).sum()) == 1 << lm
    n = 3 * CS + CS // 3 + 5
    sym = draw(rng, p, n, kind)
    msg, out = gpu_pair(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    assert int.from_bytes(ref[12:16].tobytes(), "little") == lm
    assert np.array_equal(msg, ref)
    assert np.array_equal(out, sym)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 4097])
def test_wide_edge_sizes(rlib, orc, cuda, n):
    rng = np.random.default_rng(n + 23)
    for lm in (13, 14):
        freq, p = model(rlib, "rare", lm, rng)
        sym = draw(rng, p, n, "rare")
        for N, CS in ((32, 64), (5, 33), (1, 7)):
            msg, out = gpu_pair(rlib, cuda, sym, freq, N, CS)
            assert np.array_equal(msg, orc.encode_message(sym, freq, N=N, chunk_symbols=CS))
            assert np.array_equal(out, sym)


def test_resolution_is_checked(rlib, orc, cuda):
    """A message decodes only with a model of its own resolution: the header's
    log2 M must match the table's sum."""
    import torch

    rng = np.random.default_rng(89)
    w = wl.weights_from_probs(wl.zipf_probs(200, 1.0))
    f12, f14 = rlib.rans_quantize_table(w, 12), rlib.rans_quantize_table(w, 14)
    sym = draw(rng, wl.zipf_probs(200, 1.0), 50_000, "zipf256")
    d = torch.from_numpy(orc.encode_message(sym, f14, N=32, chunk_symbols=4096)).to(cuda)
    _, st = rlib.decode(d, sym.size, f12, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    d12 = torch.from_numpy(orc.encode_message(sym, f12, N=32, chunk_symbols=4096)).to(cuda)
    _, st = rlib.decode(d12, sym.size, f14, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(st.item()) == rlib.RANS_ERR_CORRUPT
    bad = f14.copy()
    bad[0] += 1                                   # sum 2^14 + 1: no resolution
    with pytest.raises(rlib.RansError):
        rlib.encode(torch.from_numpy(sym).to(cuda), bad, 32, 4096)


def test_wide_host_paths(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(97)
    freq, p = model(rlib, "zipf256", 14, rng)
    sym = draw(rng, p, 40 << 20, "zipf256")          # two pieces
    ref = orc.encode_message(sym, freq, N=32, chunk_symbols=65536)
    m, st = rlib.encode_host(torch.from_numpy(sym).pin_memory(), freq, 32, 65536, device=cuda)
    assert st == rlib.RANS_OK and np.array_equal(m.numpy(), ref)
    out, st = rlib.decode_host(torch.from_numpy(ref).pin_memory(), sym.size, freq, 32, 65536,
                               device=cuda)
    assert st == rlib.RANS_OK and np.array_equal(out.numpy(), sym)


def test_wide_models_code_rare_symbols_closer_to_their_entropy(rlib, orc, cuda):
    """With a dominant symbol and 255 rare ones, 14 bits of resolution give
    the rare symbols probabilities closer to theirs than 12 bits can (where
    each needs at least 1/4096): the message gets smaller."""
    rng = np.random.default_rng(101)
    p = np.full(256, 1.0)
    p[0] = 4e5
    p /= p.sum()
    sym = rng.choice(256, size=1 << 20, p=p).astype(np.uint8)
    sizes = {}
    for lm in (12, 14):
        freq = rlib.rans_quantize_table(wl.weights_from_probs(p), lm)
        msg, out = gpu_pair(rlib, cuda, sym, freq, 32, 65536)
        assert np.array_equal(out, sym)
        sizes[lm] = msg.size
    assert sizes[14] < 0.9 * sizes[12], sizes
