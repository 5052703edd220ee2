"""Host-side prefix-code functions of the library (package-merge code
lengths, canonical codes, size bounds) against the oracle's -- no GPU."""
import numpy as np
import pytest


def _weights(rng, n, kind):
    if kind == "uniform":
        return rng.integers(1, 1 << 20, size=n).astype(np.uint64)
    if kind == "ties":                    # many equal weights: the tie rule decides
        return rng.integers(1, 4, size=n).astype(np.uint64)
    if kind == "skewed":                  # geometric: the length limit binds
        return (2 ** rng.integers(0, 40, size=n)).astype(np.uint64)
    if kind == "sparse":
        w = rng.integers(1, 1000, size=n).astype(np.uint64)
        w[rng.random(n) < 0.6] = 0
        if not w.any():
            w[0] = 1
        return w
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "ties", "skewed", "sparse"])
def test_lengths_and_codes_match_oracle(rlib, orc, kind):
    rng = np.random.default_rng(hash(kind) & 0xFFFF)
    for _ in range(60):
        n = int(rng.integers(1, 257))
        w = _weights(rng, n, kind)
        for max_len in (12, 9, 8):
            if np.count_nonzero(w) > (1 << max_len):
                continue
            ln = rlib.rans_prefix_lengths(w, max_len)
            assert np.array_equal(ln, orc.prefix_lengths(w, max_len)), (n, max_len)
            assert np.array_equal(rlib.rans_prefix_codes(ln).astype(np.uint32),
                                  orc.prefix_codes(ln))


def test_prefix_host_edge_cases(rlib, orc):
    assert list(rlib.rans_prefix_lengths(np.array([0, 5, 0], dtype=np.uint64))) == [0, 1, 0]
    with pytest.raises(rlib.RansError):
        rlib.rans_prefix_lengths(np.zeros(4, dtype=np.uint64))
    with pytest.raises(rlib.RansError):                     # 5 symbols cannot fit in 2 bits
        rlib.rans_prefix_lengths(np.ones(5, dtype=np.uint64), 2)
    with pytest.raises(rlib.RansError):
        rlib.rans_prefix_lengths(np.ones(4, dtype=np.uint64), 13)
    with pytest.raises(rlib.RansError):                     # Kraft sum 3/2
        rlib.rans_prefix_codes(np.array([1, 1, 1], dtype=np.uint8))
    with pytest.raises(rlib.RansError):                     # longer than 12
        rlib.rans_prefix_codes(np.array([1, 13], dtype=np.uint8))
    lengths = np.array([3, 3, 3, 3, 3, 2, 4, 4], dtype=np.uint8)
    assert list(rlib.rans_prefix_codes(lengths)) == [2, 3, 4, 5, 6, 0, 14, 15]


def test_prefix_size_bound_covers_oracle(rlib, orc):
    rng = np.random.default_rng(5)
    for N, CS, n in ((32, 4096, 20000), (7, 1001, 5000), (1, 64, 777), (32, 7, 300)):
        ln = np.full(16, 4, dtype=np.uint8)                     # 16 codes of 4 bits
        sym = rng.integers(0, 16, size=n).astype(np.uint8)
        m = orc.encode_message_prefix(sym, ln, N=N, chunk_symbols=CS)
        assert m.size <= rlib.rans_max_encoded_size_prefix(n, N, CS)
        w = np.ones(256, dtype=np.uint64)
        w[0] = 1 << 40                                          # one short code, 255 long ones
        ln = orc.prefix_lengths(w, 12)
        sym = rng.integers(1, 256, size=n).astype(np.uint8)     # the long codes only
        m = orc.encode_message_prefix(sym, ln, N=N, chunk_symbols=CS)
        assert m.size <= rlib.rans_max_encoded_size_prefix(n, N, CS)
