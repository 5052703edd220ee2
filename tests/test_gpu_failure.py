"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out ends its kernel with RANS_ERR_TIMEOUT (the barrier it waits on
is never completed; the chunk size a look-back waits for is never
published), and the context stays usable afterwards."""
import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_with_a_status(rlib, orc, cuda):
    import time

    import torch

    status = torch.zeros(1, dtype=torch.int32, device=cuda)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rlib.rans_check_bounded_wait(status)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(status.item()) == rlib.RANS_ERR_TIMEOUT
    assert 0.15 < waited < 5.0
    # the context still decodes correctly
    rng = np.random.default_rng(5)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
    sym = rng.choice(256, size=100_000, p=freq / freq.sum()).astype(np.uint8)
    msg = orc.encode_message(sym, freq, N=32, chunk_symbols=4096)
    out, st = rlib.decode(torch.from_numpy(msg).to(cuda), sym.size, freq, 32, 4096)
    assert int(st.item()) == rlib.RANS_OK
    assert np.array_equal(out.cpu().numpy(), sym)


def test_lookback_wait_gives_up_with_a_status(rlib, orc, cuda):
    """The encoder's look-back for a chunk whose predecessor never publishes
    gives up after its bound, and the context still encodes correctly."""
    import time

    import torch

    status = torch.zeros(1, dtype=torch.int32, device=cuda)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rlib.rans_check_lookback_wait(status)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(status.item()) == rlib.RANS_ERR_TIMEOUT
    assert 0.15 < waited < 5.0
    rng = np.random.default_rng(6)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(wl.zipf_probs(256, 1.1)))
    sym = rng.choice(256, size=300_000, p=freq / freq.sum()).astype(np.uint8)
    buf, size, st = rlib.encode(torch.from_numpy(sym).to(cuda), freq, 32, 4096)
    assert int(st.item()) == rlib.RANS_OK
    got = buf[: int(size.item())].cpu().numpy()
    assert np.array_equal(got, orc.encode_message(sym, freq, N=32, chunk_symbols=4096))
