"""Streams and graphs: the single-message coder captured in a CUDA graph and
replayed on new data, and several host threads coding concurrently on their
own streams -- every result checked against the oracle."""
import threading

import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_encode_and_decode_replay_in_cuda_graphs(rlib, orc, cuda):
    """rans_encode captured once, replayed on new symbols written into the
    same input buffer (the message size comes back in a device word);
    rans_decode captured once and replayed.  The first calls happen outside
    capture (they set function attributes and query occupancy)."""
    import torch

    rng = np.random.default_rng(211)
    p = wl.zipf_probs(100, 1.05)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    n, N, CS = 500_003, 32, 8192
    cap = rlib.rans_max_encoded_size(n, N, CS)
    scap = rlib.rans_encode_scratch_size(n, N, CS)
    sym = torch.empty(n, dtype=torch.uint8, device=cuda)
    msg = torch.empty(cap, dtype=torch.uint8, device=cuda)
    scratch = torch.empty(scap, dtype=torch.uint8, device=cuda)
    size = torch.zeros(1, dtype=torch.int64, device=cuda)
    est = torch.zeros(1, dtype=torch.int32, device=cuda)
    s = torch.cuda.Stream()

    def encode():
        rlib.rans_encode(sym, n, freq, N, CS, msg, cap, size, est, scratch, scap, s)

    first = wl.iid_symbols(rng, p, n)
    sym.copy_(torch.from_numpy(first))
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        encode()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            encode()
    for _ in range(2):
        data = wl.iid_symbols(rng, p, n)
        sym.copy_(torch.from_numpy(data))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert int(est.item()) == 0
        got = msg[: int(size.item())].cpu().numpy()
        assert np.array_equal(got, orc.encode_message(data, freq, N=N, chunk_symbols=CS))

    ref = orc.encode_message(first, freq, N=N, chunk_symbols=CS)
    d_msg = torch.from_numpy(ref).to(cuda)
    out = torch.empty(n, dtype=torch.uint8, device=cuda)
    dst = torch.zeros(1, dtype=torch.int32, device=cuda)

    def decode():
        rlib.rans_decode(d_msg, d_msg.numel(), freq, N, CS, out, n, dst, s)

    with torch.cuda.stream(s):
        decode()
    s.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g2, stream=s):
            decode()
    for _ in range(2):
        out.zero_()
        torch.cuda.synchronize()
        g2.replay()
        torch.cuda.synchronize()
        assert int(dst.item()) == 0
        assert np.array_equal(out.cpu().numpy(), first)


def test_host_threads_code_concurrently_on_their_streams(rlib, orc, cuda):
    """Four host threads, each on its own CUDA stream with its own lane count
    and chunk size, encode and decode three messages each at the same time;
    every message equals the oracle's and decodes back."""
    import torch

    cases = [(32, 65536), (7, 4096), (32, 1024), (1, 777)]
    errors = []
    barrier = threading.Barrier(len(cases))

    def work(k, N, CS):
        try:
            rng = np.random.default_rng(300 + k)
            p = wl.dirichlet_probs(rng, 200, 0.5)
            freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
            s = torch.cuda.Stream(cuda)
            barrier.wait()
            for it in range(3):
                data = wl.iid_symbols(rng, p, 200_000 + 7919 * it)
                with torch.cuda.stream(s):
                    d = torch.from_numpy(data).to(cuda)
                    buf, size, st = rlib.encode(d, freq, N, CS, stream=s, sync=False)
                s.synchronize()
                m = buf[: int(size.item())]
                ref = orc.encode_message(data, freq, N=N, chunk_symbols=CS)
                if int(st.item()) != 0 or not np.array_equal(m.cpu().numpy(), ref):
                    errors.append((k, it, "encode"))
                with torch.cuda.stream(s):
                    out, st = rlib.decode(m, data.size, freq, N, CS, stream=s, sync=False)
                s.synchronize()
                if int(st.item()) != 0 or not np.array_equal(out.cpu().numpy(), data):
                    errors.append((k, it, "decode"))
        except Exception as e:  # noqa: BLE001
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=work, args=(k, N, CS)) for k, (N, CS) in enumerate(cases)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
