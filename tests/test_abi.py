"""The C-ABI library without a GPU: it loads, exports every symbol that
include/rans.h declares, and its host-only logic (quantizer, size queries,
argument checks) behaves.  No call here touches a CUDA device."""
import ctypes
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "rans.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(rans_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rans_quantize_table", "rans_encode", "rans_decode"):
        assert required in names


def test_library_exports_every_declared_symbol(rlib):
    lib = ctypes.CDLL(rlib.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_status_strings(rlib):
    assert rlib.rans_version() == 1
    assert rlib.rans_status_string(0) == "ok"
    assert rlib.rans_status_string(rlib.RANS_ERR_CORRUPT) == "corrupt message"
    assert rlib.rans_status_string(999) == "unknown status"


def test_quantizer_matches_oracle(rlib, orc):
    rng = np.random.default_rng(31)
    for trial in range(400):
        n = int(rng.integers(1, 257))
        bits = int(rng.integers(1, 55))
        w = rng.integers(0, 1 << bits, size=n).astype(np.uint64)
        w[rng.random(n) < 0.25] = 0
        if not w.any():
            w[int(rng.integers(0, n))] = 1
        log2_M = 12 if trial % 3 else int(rng.integers(8, 16))
        if np.count_nonzero(w) > (1 << log2_M):
            continue
        assert np.array_equal(rlib.rans_quantize_table(w, log2_M), orc.quantize(w, log2_M))


def test_quantizer_workload_tables(rlib, orc):
    from paper_1402_3392_b300 import workloads as wl

    rng = wl.rng_for("batched")
    tables = [wl.zipf_probs(256, 1.1), wl.zipf_probs(256, 1.2)]
    tables += [wl.dirichlet_probs(rng, int(rng.integers(16, 257)), 0.3) for _ in range(50)]
    for p in tables:
        w = wl.weights_from_probs(p)
        f = rlib.rans_quantize_table(w)
        assert np.array_equal(f, orc.quantize(w))
        assert int(f.sum()) == 4096 and f.min() >= 1


def test_quantizer_rejects_bad_input(rlib):
    with pytest.raises(rlib.RansError):
        rlib.rans_quantize_table(np.zeros(4, dtype=np.uint64))
    with pytest.raises(rlib.RansError):
        rlib.rans_quantize_table(np.ones(5000, dtype=np.uint64))
    with pytest.raises(rlib.RansError):
        rlib.rans_quantize_table(np.ones(8, dtype=np.uint64), log2_M=2)   # 8 nonzero > M = 4


def test_size_queries_match_oracle(rlib, orc):
    for n, N, cs in ((0, 32, 65536), (1, 1, 1), (1 << 20, 32, 1 << 20), (1 << 30, 32, 1 << 16),
                     (12345, 7, 100)):
        assert rlib.rans_max_encoded_size(n, N, cs) == orc.max_message_size(n, N, cs)
    assert rlib.rans_max_encoded_size(10, 0, 10) == 0
    assert rlib.rans_max_encoded_size(10, 33, 10) == 0
    assert rlib.rans_encode_scratch_size(10, 32, 0) == 0
    assert rlib.rans_encode_scratch_size(1 << 30, 32, 1 << 16) >= 2 << 30


def test_argument_errors_return_without_touching_the_device(rlib):
    f = np.zeros(256, dtype=np.uint16)
    f[:] = 16
    bad_f = f.copy()
    bad_f[0] = 17
    fake = 1 << 40  # never dereferenced: every call below fails its argument checks
    E = rlib.RANS_ERR_INVALID_ARG
    assert rlib.rans_decode(fake, 4096, bad_f, 32, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(fake, 4096, f, 0, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(fake, 4095, f, 32, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(fake + 8, 4096, f, 32, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(fake, 16, f, 32, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(fake, 4096, f[:0], 32, 1024, fake, 100, fake, 0, check=False) == E
    assert rlib.rans_decode(None, 4096, f, 32, 1024, fake, 100, fake, 0, check=False) == E
    cap = rlib.rans_max_encoded_size(100, 32, 1024)
    scap = rlib.rans_encode_scratch_size(100, 32, 1024)
    assert rlib.rans_encode(fake, 100, bad_f, 32, 1024, fake, cap, fake, fake, fake, scap, 0,
                            check=False) == E
    assert rlib.rans_encode(fake, 100, f, 32, 1024, fake + 2, cap, fake, fake, fake, scap, 0,
                            check=False) == E
    assert rlib.rans_encode(fake, 100, f, 32, 1024, fake, cap - 1, fake, fake, fake, scap, 0,
                            check=False) == rlib.RANS_ERR_BUFFER_TOO_SMALL
    assert rlib.rans_encode(fake, 100, f, 32, 1024, fake, cap, fake, fake, fake, scap - 1, 0,
                            check=False) == rlib.RANS_ERR_BUFFER_TOO_SMALL
    # worst case beyond 4 GiB of chunk data (u32 offsets)
    big = 3 << 30
    assert rlib.rans_encode(fake, big, f, 32, 65536, fake, 1 << 62, fake, fake, fake, 1 << 62, 0,
                            check=False) == E


def test_package_imports_without_building_the_oracle():
    import paper_1402_3392_b300.rans as r
    import sys

    assert "oracle" not in getattr(r, "__dict__", {})
    src = open(r.__file__).read() + open(os.path.join(os.path.dirname(r.__file__),
                                                      "workloads.py")).read()
    assert "import oracle" not in src and "from oracle" not in src
