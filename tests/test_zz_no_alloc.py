"""rans_encode_static_scratch: the encoder for callers that cannot allocate
device memory (for example a host that reserved the device up front, or a
real-time pipeline that forbids allocation while it runs).  Its scratch is a
fixed array inside the library instead of a caller buffer.

The test calls it through the C ABI several times in a row, with different
inputs and models (12- and 14-bit), and checks each message byte for byte
(the coder's tolerance is zero) against the CPU oracle's message and against
the ordinary rans_encode on the same input.  It also checks that an input
whose scratch need is above the fixed array's size is refused without
launching.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _encode_both(rlib, torch, dev, sym, freq, N, CS):
    n = sym.numel()
    cap = rlib.rans_max_encoded_size(n, N, CS)
    out_a = torch.empty(cap, dtype=torch.uint8, device=dev)
    out_b = torch.empty(cap, dtype=torch.uint8, device=dev)
    size_a = torch.zeros(1, dtype=torch.int64, device=dev)
    size_b = torch.zeros(1, dtype=torch.int64, device=dev)
    st_a = torch.ones(1, dtype=torch.int32, device=dev)
    st_b = torch.ones(1, dtype=torch.int32, device=dev)
    scap = rlib.rans_encode_scratch_size(n, N, CS)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    rlib.rans_encode(sym, n, freq, N, CS, out_a, cap, size_a, st_a, scratch, scap)
    rlib.rans_encode_static_scratch(sym, n, freq, N, CS, out_b, cap, size_b, st_b)
    torch.cuda.synchronize(dev)
    assert int(st_a.item()) == 0 and int(st_b.item()) == 0
    sa, sb = int(size_a.item()), int(size_b.item())
    assert sa == sb and sa > 0
    return out_a[:sa], out_b[:sb]


def test_static_scratch_encode_matches_oracle_and_rans_encode(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(71)
    cases = [
        (wl.zipf_probs(256, 1.1), 3 * 65536 + 4321, 32, 65536, 12),
        (wl.dirichlet_probs(rng, 97, 0.3), 200_001, 7, 1000, 12),
        (wl.zipf_probs(256, 1.3), 150_003, 32, 4096, 14),
    ]
    for p, n, N, CS, lm in cases:          # calls in a row on the shared array
        freq = rlib.rans_quantize_table(wl.weights_from_probs(p), lm)
        h_sym = wl.iid_symbols(rng, p, n)
        sym = torch.from_numpy(h_sym).to(cuda)
        a, b = _encode_both(rlib, torch, cuda, sym, freq, N, CS)
        ref = orc.encode_message(h_sym, freq, N=N, chunk_symbols=CS)
        assert np.array_equal(b.cpu().numpy(), ref)
        assert torch.equal(a, b)
        out, _ = rlib.decode(b, n, freq, N, CS)
        assert torch.equal(out, sym)


def test_static_scratch_refuses_inputs_above_its_size(rlib, cuda):
    import torch

    N, CS = 32, 65536
    n = 1
    while rlib.rans_encode_scratch_size(n, N, CS) <= rlib.RANS_STATIC_SCRATCH_BYTES:
        n *= 2
    freq = np.full(256, 16, dtype=np.uint16)
    cap = rlib.rans_max_encoded_size(n, N, CS)
    out = torch.empty(cap, dtype=torch.uint8, device=cuda)
    size = torch.zeros(1, dtype=torch.int64, device=cuda)
    st = torch.full((1,), 99, dtype=torch.int32, device=cuda)
    sym = torch.zeros(n, dtype=torch.uint8, device=cuda)
    rc = rlib.rans_encode_static_scratch(sym, n, freq, N, CS, out, cap, size, st, check=False)
    assert rc == rlib.RANS_ERR_BUFFER_TOO_SMALL
    torch.cuda.synchronize()
    assert int(st.item()) == 99                 # nothing was enqueued
