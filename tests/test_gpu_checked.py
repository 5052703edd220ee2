"""The checked build (-DRANS_CHECKED) on the GPU: the kernels test their
invariants as they run -- the decoder's TMA ring never reads a segment
before its copy completes or after a later copy took its slot, the encoders'
stores stay inside their slots -- and count the failures.  A child process
loads that build, makes one check fail on purpose (the counter must see it),
then runs every message kind, the batched coder and the host-memory paths
against the oracle, and must end with no failed check."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_1402_3392_b300 import rans, batch as B, workloads as wl

assert rans.library_path().endswith("_checked.so"), rans.library_path()
orc = oracle.default()
dev = torch.device("cuda:0")
assert rans.rans_debug_checks() == 0
rans.rans_debug_check_selftest()
assert rans.rans_debug_checks() == 1, "the deliberate failure was not counted"

rng = np.random.default_rng(5)
p = wl.zipf_probs(256, 1.1)
freq = rans.rans_quantize_table(wl.weights_from_probs(p))
def d(a): return torch.from_numpy(a).to(dev)

# plain: one chunk per warp, and two per warp (more than 5x the resident warps)
for n, N, CS in ((400_003, 32, 4096), (777, 5, 33), (24_000 * 1024 + 77, 32, 1024)):
    sym = wl.iid_symbols(rng, p, n)
    m, _, _ = rans.encode(d(sym), freq, N, CS)
    assert np.array_equal(m.cpu().numpy(), orc.encode_message(sym, freq, N=N, chunk_symbols=CS))
    out, _ = rans.decode(m, n, freq, N, CS)
    assert np.array_equal(out.cpu().numpy(), sym)
sym = wl.iid_symbols(rng, p, 300_007)
flags = (np.arange(256) >= 16).astype(np.uint8)
raw = rng.integers(0, 1 << 16, size=sym.size).astype(np.uint16)
m, _, _ = rans.encode_bypass(d(sym), d(raw.view(np.int16)), freq, flags, 32, 4096)
assert np.array_equal(m.cpu().numpy(), orc.encode_message_bypass(sym, raw, freq, flags, N=32,
                                                                  chunk_symbols=4096))
o, r, _ = rans.decode_bypass(m, sym.size, freq, flags, 32, 4096)
assert np.array_equal(o.cpu().numpy(), sym)
m, _, _ = rans.encode_bytes(d(sym), freq, 7, 4096)
assert np.array_equal(m.cpu().numpy(), orc.encode_message_bytes(sym, freq, N=7, chunk_symbols=4096))
o, _ = rans.decode_bytes(m, sym.size, freq, 7, 4096)
assert np.array_equal(o.cpu().numpy(), sym)
bits = wl.drifting_bits(rng, 300_007, 4096)
m, _, _ = rans.encode_adaptive(d(bits), 32, 4096)
assert np.array_equal(m.cpu().numpy(), orc.encode_message_adaptive(bits, N=32, chunk_symbols=4096))
o, _ = rans.decode_adaptive(m, bits.size, 32, 4096)
assert np.array_equal(o.cpu().numpy(), bits)
ln = orc.prefix_lengths(wl.weights_from_probs(p), 12)
m, _, _ = rans.encode_prefix(d(sym), ln, 32, 4096)
assert np.array_equal(m.cpu().numpy(), orc.encode_message_prefix(sym, ln, N=32, chunk_symbols=4096))
o, _ = rans.decode_prefix(m, sym.size, ln, 32, 4096)
assert np.array_equal(o.cpu().numpy(), sym)

# batched coder: 200 streams of mixed sizes, one model each
sizes = wl.log_uniform_sizes(rng, 200, 1 << 10, 1 << 18)
tables = [rans.rans_quantize_table(wl.weights_from_probs(wl.dirichlet_probs(rng, 64, 0.3)))
          for _ in range(200)]
syms = [rng.choice(64, size=int(s), p=t / t.sum()).astype(np.uint8) for s, t in zip(sizes, tables)]
offs, total = B.aligned_offsets(sizes)
arena = torch.zeros(total, dtype=torch.uint8, device=dev)
for o_, s_ in zip(offs, syms):
    arena[o_:o_ + s_.size] = d(s_)
tdev = B.upload_tables(tables, dev)
n_sym = [s_.size for s_ in syms]
eb = B.encode_batch(arena, offs, n_sym, tdev, list(range(200)), 32, 16384)
torch.cuda.synchronize()
assert not eb.status.any()
for i in (0, 57, 199):
    ref = orc.encode_message(syms[i], tables[i], N=32, chunk_symbols=16384)
    assert np.array_equal(eb.message(i).cpu().numpy(), ref), i
dec = B.BatchDecoder(eb.arena, eb.offsets, eb.host_sizes(), n_sym, tdev, list(range(200)), 32,
                     16384)
st = dec()
torch.cuda.synchronize()
assert not st.any()
for i, o_ in enumerate(offs):
    assert torch.equal(dec.output(i), arena[o_:o_ + n_sym[i]]), i

# host-memory paths, two pieces each
big = wl.iid_symbols(rng, p, 40 << 20)
hs = torch.from_numpy(big).pin_memory()
m, st = rans.encode_host(hs, freq, 32, 65536, device=dev)
ref = orc.encode_message(big, freq, N=32, chunk_symbols=65536)
assert st == 0 and np.array_equal(m.numpy(), ref)
out, st = rans.decode_host(torch.from_numpy(ref).pin_memory(), big.size, freq, 32, 65536,
                           device=dev)
assert st == 0 and np.array_equal(out.numpy(), big)

print("failed checks:", rans.rans_debug_checks())
'''


def test_checked_build_holds_its_invariants(rlib):
    from paper_1402_3392_b300 import build

    build.build(checked=True)
    env = dict(os.environ, RANS_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT), 1)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.strip().splitlines()[-1] == "failed checks: 0", r.stdout[-2000:]


def test_normal_build_has_no_checks(rlib):
    with pytest.raises(rlib.RansError):
        rlib.rans_debug_checks()
