"""The continuous-batching server (rans_server_*): every request's result in
a mixed, overlapping trace is byte-identical to the oracle's and to the same
request served alone; admission respects arrival times and the memory
budget; a request that can never fit fails alone with RANS_ERR_OOM."""
import numpy as np
import pytest

from paper_1402_3392_b300 import batch as B
from paper_1402_3392_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def make_trace(rlib, orc, torch, rng, count, rate, size_hi=1 << 20):
    sizes = wl.log_uniform_sizes(rng, count, 4 << 10, size_hi)
    probs = wl.batched_models(rng, count, 64, 256, 0.5)
    tables = [rlib.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    arrivals = wl.poisson_arrivals(rng, rate, count)
    kinds = rng.integers(0, 2, size=count)
    reqs = np.zeros(count, dtype=rlib.REQUEST_DTYPE)
    keep, expect = [], []
    for i in range(count):
        f = tables[i]
        sym = rng.choice(len(f), size=int(sizes[i]), p=f / f.sum()).astype(np.uint8)
        msg = orc.encode_message(sym, f, N=32, chunk_symbols=16384)
        if kinds[i] == rlib.RANS_REQ_ENCODE:
            inp, exp, cap = sym, msg, rlib.rans_max_encoded_size(sym.size, 32, 16384)
        else:
            inp, exp, cap = msg, sym, sym.size
        h_in = torch.from_numpy(inp.copy()).pin_memory()
        h_out = torch.zeros(max(cap, 1), dtype=torch.uint8).pin_memory()
        keep += [h_in, h_out]
        expect.append(exp)
        reqs[i] = (kinds[i], i, 32, 16384, h_in.data_ptr(), inp.size, sym.size, h_out.data_ptr(),
                   cap, arrivals[i])
    return reqs, tables, keep, expect


def out_bytes(reqs, res, i):
    import ctypes

    n = int(res["output_size"][i])
    return np.ctypeslib.as_array((ctypes.c_uint8 * max(n, 1)).from_address(int(reqs["output"][i])))[:n].copy()


def test_mixed_trace_is_exact_and_batches_overlap(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(131)
    reqs, tables, keep, expect = make_trace(rlib, orc, torch, rng, 80, rate=3000.0)
    tdev = B.upload_tables(tables, cuda)
    arena = torch.empty(24 << 20, dtype=torch.uint8, device=cuda)   # small budget: admission waits
    srv = rlib.Server(tdev, arena, max_batch=16, n_slots=3)
    res = srv.run(reqs)
    assert (res["status"] == 0).all(), res["status"]
    for i in range(reqs.size):
        assert np.array_equal(out_bytes(reqs, res, i), expect[i]), i
    assert (res["admit_s"] >= reqs["arrival_s"] - 1e-9).all()
    assert (res["done_s"] >= res["admit_s"]).all()
    assert len(set(res["batch"].tolist())) > 3            # served in several batches
    # some batch was admitted while an earlier one was still running
    order = np.argsort(res["admit_s"])
    overlaps = 0
    for a, b in zip(order[:-1], order[1:]):
        if res["batch"][a] != res["batch"][b] and res["admit_s"][b] < res["done_s"][a]:
            overlaps += 1
    assert overlaps > 0
    # the same requests served alone give the same bytes
    for i in rng.choice(reqs.size, size=6, replace=False):
        one = reqs[i:i + 1].copy()
        one["arrival_s"] = 0.0
        torch.from_numpy(np.zeros(int(one["output_cap"][0]), dtype=np.uint8))  # noqa: B018
        r1 = srv.run(one)
        assert r1["status"][0] == 0
        assert np.array_equal(out_bytes(one, r1, 0), expect[i]), i
    srv.close()


def test_request_that_never_fits_fails_alone(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(137)
    reqs, tables, keep, expect = make_trace(rlib, orc, torch, rng, 10, rate=1000.0, size_hi=64 << 10)
    big = np.zeros(1, dtype=rlib.REQUEST_DTYPE)
    h_in = torch.zeros(3 << 20, dtype=torch.uint8).pin_memory()
    h_out = torch.zeros(rlib.rans_max_encoded_size(3 << 20, 32, 16384), dtype=torch.uint8).pin_memory()
    big[0] = (rlib.RANS_REQ_ENCODE, 0, 32, 16384, h_in.data_ptr(), h_in.numel(), h_in.numel(),
              h_out.data_ptr(), h_out.numel(), 0.0)
    trace = np.concatenate([big, reqs])
    trace["arrival_s"][0] = 0.0
    tdev = B.upload_tables(tables, cuda)
    arena = torch.empty(4 << 20, dtype=torch.uint8, device=cuda)
    srv = rlib.Server(tdev, arena, max_batch=8, n_slots=2)
    res = srv.run(trace)
    assert res["status"][0] == rlib.RANS_ERR_OOM
    assert (res["status"][1:] == 0).all()
    for i in range(reqs.size):
        assert np.array_equal(out_bytes(trace, res, i + 1), expect[i]), i
    srv.close()


def test_device_resident_requests_equal_oracle(rlib, orc, cuda):
    """Requests flagged RANS_REQ_DEVICE_MEMORY read their input from and write
    their output to device buffers in place (no copies; the arena holds only
    the batches' scratch).  In a trace that mixes them with host-payload
    requests, every result equals the oracle's."""
    import torch

    rng = np.random.default_rng(149)
    count = 60
    sizes = wl.log_uniform_sizes(rng, count, 4 << 10, 4 << 20)
    probs = wl.batched_models(rng, count, 64, 256, 0.5)
    tables = [rlib.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    arrivals = wl.poisson_arrivals(rng, 5000.0, count)
    kinds = rng.integers(0, 2, size=count)
    on_dev = rng.integers(0, 2, size=count).astype(bool)
    reqs = np.zeros(count, dtype=rlib.REQUEST_DTYPE)
    keep, expect, outs = [], [], []
    for i in range(count):
        f = tables[i]
        sym = rng.choice(len(f), size=int(sizes[i]), p=f / f.sum()).astype(np.uint8)
        msg = orc.encode_message(sym, f, N=32, chunk_symbols=16384)
        if kinds[i] == rlib.RANS_REQ_ENCODE:
            inp, exp, cap = sym, msg, rlib.rans_max_encoded_size(sym.size, 32, 16384)
        else:
            inp, exp, cap = msg, sym, sym.size
        if on_dev[i]:
            b_in = torch.from_numpy(inp.copy()).to(cuda)
            b_out = torch.zeros(max(cap, 16), dtype=torch.uint8, device=cuda)
            kind = int(kinds[i]) | rlib.RANS_REQ_DEVICE_MEMORY
        else:
            b_in = torch.from_numpy(inp.copy()).pin_memory()
            b_out = torch.zeros(max(cap, 1), dtype=torch.uint8).pin_memory()
            kind = int(kinds[i])
        keep += [b_in, b_out]
        outs.append(b_out)
        expect.append(exp)
        reqs[i] = (kind, i, 32, 16384, b_in.data_ptr(), inp.size, sym.size, b_out.data_ptr(),
                   cap, arrivals[i])
    tdev = B.upload_tables(tables, cuda)
    arena = torch.empty(64 << 20, dtype=torch.uint8, device=cuda)
    srv = rlib.Server(tdev, arena, max_batch=16, n_slots=3)
    res = srv.run(reqs)
    srv.close()
    assert (res["status"] == 0).all(), res["status"]
    for i in range(count):
        n_out = int(res["output_size"][i])
        got = outs[i][:n_out].cpu().numpy()
        assert n_out == expect[i].size and np.array_equal(got, expect[i]), (i, bool(on_dev[i]))
