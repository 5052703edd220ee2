"""CUDA path vs the CPU oracle, byte for byte (zero tolerance: the coder is
integer arithmetic and the bitstream is unique, Sections 3 and 5).

Every call goes through the C ABI (ctypes binding); inputs are seeded and
synthetic (paper_1402_3392_b300.workloads)."""
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
    elif kind == "zipf200":
        p = wl.zipf_probs(200, 1.2)
    elif kind == "dirichlet":
        p = wl.dirichlet_probs(rng, int(rng.integers(16, 257)), 0.3)
    elif kind == "binary":
        p0 = float(rng.uniform(0.5, 0.999))
        p = np.array([p0, 1 - p0])
    elif kind == "binary_extreme":
        p = np.array([1 - 1e-9, 1e-9])
    elif kind == "uniform256":
        p = np.full(256, 1 / 256)
    elif kind == "single":
        p = np.array([1.0])
    elif kind == "rare_heavy":     # many f = 1 symbols, drawn often
        p = np.full(200, 1.0)
        p[0] = 1e6
        p /= p.sum()
    else:
        raise ValueError(kind)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    return freq


def draw(rng, freq, n, kind):
    q = freq / freq.sum()
    if kind == "rare_heavy":
        return rng.integers(0, len(freq), size=n).astype(np.uint8)
    return rng.choice(len(freq), size=n, p=q).astype(np.uint8)


def gpu_roundtrip(rlib, cuda, sym, freq, N, CS):
    import torch

    d = torch.from_numpy(sym).to(cuda) if sym.size else torch.empty(0, dtype=torch.uint8,
                                                                      device=cuda)
    msg, _, _ = rlib.encode(d, freq, N, CS)
    out, _ = rlib.decode(msg, sym.size, freq, N, CS)
    return msg.cpu().numpy(), out.cpu().numpy()


CASES = list(itertools.product(
    ["zipf256", "dirichlet", "binary", "uniform256", "single", "rare_heavy"],
    [32, 1, 5, 16, 31],
    [4096, 1000, 65536],
))


@pytest.mark.parametrize("kind,N,CS", CASES)
def test_bitstream_matches_oracle(rlib, orc, cuda, kind, N, CS):
    rng = np.random.default_rng(zlib.crc32(repr((kind, N, CS)).encode()))
    freq = model(rlib, kind, rng)
    # several chunks and a ragged tail: the last chunk and the last step are partial
    n = 3 * CS + CS // 3 + 7 if CS <= 4096 else CS + 12345
    sym = draw(rng, freq, n, kind)
    msg, back = gpu_roundtrip(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    assert msg.size == ref.size
    assert np.array_equal(msg, ref)
    assert np.array_equal(back, sym)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 63, 64, 65, 255, 256, 257, 4095, 4097])
@pytest.mark.parametrize("N,CS", [(32, 64), (32, 4096), (7, 33), (1, 5), (32, 1)])
def test_edge_sizes(rlib, orc, cuda, n, N, CS):
    rng = np.random.default_rng(n * 1000 + N * 10 + CS)
    freq = model(rlib, "zipf200", rng)
    sym = draw(rng, freq, n, "zipf200")
    msg, back = gpu_roundtrip(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(back, sym)


def test_long_chunk_many_segments(rlib, orc, cuda):
    """One chunk whose word stream spans hundreds of ring segments,
    for the least compressible (uniform) and a skewed model."""
    rng = np.random.default_rng(41)
    for kind in ("uniform256", "zipf256", "binary_extreme"):
        freq = model(rlib, kind, rng)
        sym = draw(rng, freq, 200_003, kind)
        msg, back = gpu_roundtrip(rlib, cuda, sym, freq, 32, 1 << 20)
        assert np.array_equal(msg, orc.encode_message(sym, freq, N=32, chunk_symbols=1 << 20))
        assert np.array_equal(back, sym)


@pytest.mark.parametrize("n_chunks,N,CS", [(9473, 32, 64), (30001, 32, 48), (25001, 7, 61)])
def test_more_chunks_than_resident_warps(rlib, orc, cuda, n_chunks, N, CS):
    """Messages with thousands of short chunks: several waves of one chunk
    per warp, and (at more than five waves of the 4736 warps a B300 holds)
    warps decoding two chunks side by side, where an odd chunk count leaves
    one warp a single chunk.  The last chunk is ragged.  A corrupt word in
    the first or the second chunk of a pair is reported."""
    import torch

    rng = np.random.default_rng(n_chunks + N)
    freq = model(rlib, "zipf256", rng)
    n = (n_chunks - 1) * CS + CS // 2 + 1
    sym = draw(rng, freq, n, "zipf256")
    msg, back = gpu_roundtrip(rlib, cuda, sym, freq, N, CS)
    ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    assert np.array_equal(msg, ref)
    assert np.array_equal(back, sym)
    offs = ref[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    for c in (n_chunks // 2, n_chunks // 2 + 1):
        bad = ref.copy()
        last_word = data0 + int(offs[c + 1]) - 2
        assert last_word >= data0 + int(offs[c]) + 4 * N   # the chunk has words
        bad[last_word] ^= 0x01
        with pytest.raises(oracle.OracleError):
            orc.decode_message(bad, n, freq, N=N, chunk_symbols=CS)
        _, status = rlib.decode(torch.from_numpy(bad).to(cuda), n, freq, N, CS, sync=False)
        torch.cuda.synchronize()
        assert int(status.item()) == rlib.RANS_ERR_CORRUPT, c


# Chunk counts on both sides of the single-message decoder's launch shapes on
# a B300 (148 SMs, 4 CTAs of 8 warps each): the entry-ahead step up to two
# chunks per SM (296), the early-word step up to half a wave of 8-warp CTAs
# (2368 chunks), the plain step in 8-warp CTAs below a wave (4736), 12-warp
# CTAs from there.  (The encoder's latency form covers up to 4736 chunks; a
# message of at most one wave of the encoder's warps takes the CTA size that
# loads the busiest SM least: 1 warp for up to 148 chunks, 4 for 592, 7 for
# 1036, 5 for 2960.)
@pytest.mark.parametrize("n_chunks,N", [(1, 32), (148, 32), (296, 32), (297, 32), (2367, 32),
                                        (2368, 32), (2369, 32), (4735, 32), (4736, 32),
                                        (4737, 32), (16, 32), (592, 32), (1036, 32),
                                        (1037, 32), (2960, 32), (296, 7), (297, 7), (2368, 7),
                                        (2369, 7),
                                        (4736, 7)])
def test_every_launch_shape(rlib, orc, cuda, n_chunks, N):
    """A message of n_chunks chunks of 96 symbols (the last one ragged) is
    bit-exact with the oracle and decodes back, whichever kernel shape the
    decoder launches for it."""
    CS = 96
    rng = np.random.default_rng(n_chunks * 100 + N)
    freq = model(rlib, "zipf256", rng)
    sym = draw(rng, freq, (n_chunks - 1) * CS + 37, "zipf256")
    msg, back = gpu_roundtrip(rlib, cuda, sym, freq, N, CS)
    assert np.array_equal(msg, orc.encode_message(sym, freq, N=N, chunk_symbols=CS))
    assert np.array_equal(back, sym)


def test_decodes_oracle_messages(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(43)
    freq = model(rlib, "dirichlet", rng)
    sym = draw(rng, freq, 50_000, "dirichlet")
    for N, CS in ((32, 4096), (3, 777)):
        ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
        out, _ = rlib.decode(torch.from_numpy(ref).to(cuda), sym.size, freq, N, CS)
        assert np.array_equal(out.cpu().numpy(), sym)


def test_encode_is_deterministic_and_stream_ordered(rlib, cuda):
    import torch

    rng = np.random.default_rng(47)
    freq = model(rlib, "zipf256", rng)
    sym = torch.from_numpy(draw(rng, freq, 1 << 20, "zipf256")).to(cuda)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a, _, _ = rlib.encode(sym, freq, 32, 4096, stream=s)
        b, _, _ = rlib.encode(sym, freq, 32, 4096, stream=s)
        out, _ = rlib.decode(a, sym.numel(), freq, 32, 4096, stream=s)
    assert torch.equal(a, b)
    assert torch.equal(out, sym)


def test_zero_frequency_symbol_is_reported(rlib, cuda):
    import torch

    freq = np.zeros(256, dtype=np.uint16)
    freq[:128] = 32
    sym = torch.full((10_000,), 5, dtype=torch.uint8, device=cuda)
    sym[1234] = 200                      # f = 0
    with pytest.raises(rlib.RansError) as e:
        rlib.encode(sym, freq, 32, 4096)
    assert e.value.code == rlib.RANS_ERR_ZERO_FREQ
    f100 = np.full(100, 41, dtype=np.uint16)
    f100[96:] = 40                       # 100 symbols, sum 4096: symbol 200 >= n_alpha
    _, size, status = rlib.encode(sym, f100, 32, 4096, sync=False)
    torch.cuda.synchronize()
    assert int(status.item()) == rlib.RANS_ERR_ZERO_FREQ and int(size.item()) == 0


def corruptions(ref, n_chunks, rng):
    """Host-side damaged copies of a message (never a device fault)."""
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = ref[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)
    out = []
    m = ref.copy(); m[0] ^= 1; out.append(("magic", m))
    m = ref.copy(); m[8] ^= 1; out.append(("lanes", m))
    m = ref.copy(); m[16] ^= 1; out.append(("n_symbols", m))
    m = ref.copy(); m[32 + 4] ^= 0x40; out.append(("offset", m))
    m = ref.copy(); m[32 + 8] ^= 0x01; out.append(("offset_odd", m))
    for k in range(6):                   # flip one bit of a word
        c = int(rng.integers(0, n_chunks))
        a, z = data0 + offs[c] + 4 * 32, data0 + offs[c + 1]
        if z > a:
            m = ref.copy()
            m[int(rng.integers(a, z))] ^= 1 << int(rng.integers(0, 8))
            out.append((f"word{k}", m))
    m = ref.copy(); c = 1; m[data0 + offs[c] + 3] = 0; out.append(("state<L", m))
    m = ref.copy(); c = 2
    m[data0 + offs[c]:data0 + offs[c] + 4] = m[data0 + offs[c] + 4:data0 + offs[c] + 8]
    out.append(("state_swap", m))
    return out


def test_corrupt_messages_are_reported_like_the_oracle(rlib, orc, cuda):
    import torch

    rng = np.random.default_rng(53)
    freq = model(rlib, "zipf256", rng)
    N, CS = 32, 4096
    sym = draw(rng, freq, 20 * CS, "zipf256")
    ref = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    for name, bad in corruptions(ref, 20, rng):
        try:
            orc.decode_message(bad, sym.size, freq, N=N, chunk_symbols=CS)
            oracle_ok = True
        except Exception:
            oracle_ok = False
        _, status = rlib.decode(torch.from_numpy(bad).to(cuda), sym.size, freq, N, CS,
                                sync=False)
        torch.cuda.synchronize()
        st = int(status.item())
        assert st in (rlib.RANS_OK, rlib.RANS_ERR_CORRUPT), name
        assert (st == rlib.RANS_OK) == oracle_ok, name
    # the untouched message still decodes
    out, _ = rlib.decode(torch.from_numpy(ref).to(cuda), sym.size, freq, N, CS)
    assert np.array_equal(out.cpu().numpy(), sym)


def test_wrong_size_or_model_is_an_argument_error(rlib, cuda):
    import torch

    freq = np.full(256, 16, dtype=np.uint16)
    msg = torch.zeros(4096, dtype=torch.uint8, device=cuda)
    out = torch.empty(100, dtype=torch.uint8, device=cuda)
    st = torch.zeros(1, dtype=torch.int32, device=cuda)
    assert rlib.rans_decode(msg, 4008, freq, 32, 64, out, 100, st, check=False) == \
        rlib.RANS_ERR_INVALID_ARG
    bad = freq.copy(); bad[3] = 0
    assert rlib.rans_decode(msg, 4096, bad, 32, 64, out, 100, st, check=False) == \
        rlib.RANS_ERR_INVALID_ARG


@pytest.mark.parametrize("workload", ["single"])
def test_full_size_workload_full_parity(rlib, orc, cuda, workload):
    """The 1 MiB single-stream workload, checked in full against the oracle."""
    import torch

    cfg = wl.WORKLOADS[workload]
    rng = wl.rng_for(workload)
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    sym = wl.iid_symbols(rng, p, cfg["n_symbols"])
    d = torch.from_numpy(sym).to(cuda)
    msg, _, _ = rlib.encode(d, freq, cfg["n_lanes"], cfg["chunk_symbols"])
    ref = orc.encode_message(sym, freq, N=cfg["n_lanes"], chunk_symbols=cfg["chunk_symbols"])
    assert np.array_equal(msg.cpu().numpy(), ref)
    out, _ = rlib.decode(msg, sym.size, freq, cfg["n_lanes"], cfg["chunk_symbols"])
    assert torch.equal(out, d)


def test_full_size_chunked_sampled_parity(rlib, orc, cuda):
    """The 1 GiB workload (16384 chunks of 64 KiB, 32 coders each) in the
    launch configuration the benchmark times: full round trip on the device,
    and sampled chunks re-encoded and decoded by the oracle one by one."""
    import torch

    cfg = wl.WORKLOADS["chunked"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    n, N, CS = cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    d = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), cuda)
    msg, _, _ = rlib.encode(d, freq, N, CS)
    out, _ = rlib.decode(msg, n, freq, N, CS)
    assert torch.equal(out, d)
    n_chunks = n // CS
    head = msg[: 32 + 4 * (n_chunks + 1)].cpu().numpy()
    h = head[:32].view(np.uint32)
    assert list(h[:4]) == [0x534E4152, 1, N, 12] and list(h[6:8]) == [CS, n_chunks]
    offs = head[32:].view(np.uint32).astype(np.int64)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    assert msg.numel() == data0 + (offs[-1] + 15) // 16 * 16
    rng = np.random.default_rng(59)
    picks = sorted({0, 1, n_chunks - 1, *rng.integers(0, n_chunks, size=5).tolist()})
    for c in picks:
        chunk_sym = d[c * CS:(c + 1) * CS].cpu().numpy()
        gpu_chunk = msg[data0 + offs[c]: data0 + offs[c + 1]].cpu().numpy()
        assert np.array_equal(gpu_chunk, orc.encode_chunk(chunk_sym, freq, N=N)), c
        assert np.array_equal(orc.decode_chunk(gpu_chunk, CS, freq, N=N), chunk_sym), c


def test_largest_message_the_format_holds(rlib, orc, cuda):
    """Offsets are u32, so with N = 32 and 64 Ki-symbol chunks a message holds
    at most 32736 chunks (its worst-case data region, 128 bytes of states a
    chunk plus 2 bytes a symbol, must stay below 2^32 - 16): that size round
    trips, sampled chunks equal the oracle's, and one chunk more is refused
    before anything runs."""
    import torch

    N, CS = 32, 1 << 16
    k_max = (0xFFFFFFF0 // (4 * N + 2 * CS))
    assert (4 * N + 2 * CS) * (k_max + 1) > 0xFFFFFFF0
    n = k_max * CS
    p = wl.zipf_probs(256, 1.1)
    freq = rlib.rans_quantize_table(wl.weights_from_probs(p))
    d = wl.iid_symbols_device(p, n, wl.seed_for("chunked", 7), cuda)
    msg, _, _ = rlib.encode(d, freq, N, CS)
    out, _ = rlib.decode(msg, n, freq, N, CS)
    assert torch.equal(out, d)
    del out
    head = msg[: 32 + 4 * (k_max + 1)].cpu().numpy()
    offs = head[32:].view(np.uint32).astype(np.int64)
    data0 = (32 + 4 * (k_max + 1) + 15) // 16 * 16
    for c in (0, k_max // 2, k_max - 1):
        chunk_sym = d[c * CS:(c + 1) * CS].cpu().numpy()
        gpu_chunk = msg[data0 + offs[c]: data0 + offs[c + 1]].cpu().numpy()
        assert np.array_equal(gpu_chunk, orc.encode_chunk(chunk_sym, freq, N=N)), c
    del msg
    torch.cuda.empty_cache()
    # One chunk more: refused by the size limit, which the library checks
    # before the buffer capacities (given as 0 here, so no launch can follow
    # whatever the answer).
    n2 = n + CS
    st = torch.zeros(1, dtype=torch.int32, device=cuda)
    size = torch.zeros(1, dtype=torch.int64, device=cuda)
    tiny = torch.empty(16, dtype=torch.uint8, device=cuda)
    assert rlib.rans_encode(d, n2, freq, N, CS, tiny, 0, size, st, tiny, 0,
                            check=False) == rlib.RANS_ERR_INVALID_ARG
