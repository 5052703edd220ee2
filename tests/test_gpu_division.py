"""The encoders' exact division, exhaustively on the GPU.

C(s, x) = floor(x / f_s) * M + B_s + (x mod f_s) (Section 2) needs the
quotient exactly.  The static encoders take it from a multiply-high by a
precomputed reciprocal, the adaptive encoder from a float estimate and one
correction.  rans_check_division runs the encoders' own division code over
every frequency f in [1, M - 1] and every state x of the precursor set
I_s = [f L / M, f b L / M) the encoder divides (L = b = 2^16), and checks
q * f <= x < (q + 1) * f in 64 bits -- the definition of floor(x / f)."""
import pytest

pytestmark = pytest.mark.gpu


def reachable_states(log2m):
    M = 1 << log2m
    return sum((f << (32 - log2m)) - (f << (16 - log2m)) for f in range(1, M))


@pytest.mark.parametrize("method,log2m", [(0, 12), (0, 13), (0, 14), (1, 12)])
def test_division_is_exact_for_every_reachable_state(rlib, cuda, method, log2m):
    import torch

    out = torch.zeros(4, dtype=torch.int64, device=cuda)
    rlib.rans_check_division(method, log2m, out)
    torch.cuda.synchronize()
    checked, wrong, first, _ = (int(v) & ((1 << 64) - 1) for v in out.cpu().tolist())
    print(f"method {method}, M = 2^{log2m}: {checked} states checked, {wrong} wrong")
    assert checked == reachable_states(log2m)
    assert wrong == 0, (first >> 32, first & 0xFFFFFFFF)
