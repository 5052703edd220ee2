"""The placing encoders' CTA-size rule (rans_check_cta_warps) -- host logic,
no GPU.  A message whose chunks all start at once is done when the SM given
the most warps is; the rule picks, of CTAs of 1 .. 8 warps, the size that
gives that SM the fewest, the larger of equal ones."""
import itertools

import numpy as np
import pytest

SMS = 148


def per_sm_table(regs, max_warps=8, smem_base=4096 + 4096 + 64 + 1024, ring=4096):
    """w-warp CTAs an SM of 64 Ki registers and 228 KiB of shared memory holds
    (the encoder's layout: table, ring alignment slack and CTA words, one 4 KiB
    ring per warp, 1 KiB reserved per CTA), at most 32 CTAs."""
    t = [0]
    for w in range(1, max_warps + 1):
        by_regs = 65536 // (regs * 32 * w)
        by_smem = 233472 // (smem_base + w * ring)
        t.append(min(by_regs, by_smem, 32))
    return t


def busiest(n, w, sms=SMS):
    return -(-(-(-n // w)) // sms) * w


# Chunk counts of the placing encoder's measured launches (80 registers a
# thread) and the CTA size each one takes.
@pytest.mark.parametrize("n,expect", [(1, 1), (16, 1), (148, 1), (592, 4), (1036, 7), (1037, 8),
                                      (2368, 8), (2960, 5), (3552, 8), (4736, 8), (100000, 8)])
def test_measured_launches(rlib, n, expect):
    assert rlib.rans_check_cta_warps(n, SMS, per_sm_table(80), 8) == expect


def test_adaptive_n_launch(rlib):
    # 4096 chunks of the 16-symbol adaptive workload, 64 registers a thread:
    # 8-warp CTAs leave some SMs 32 warps and others 24; 7-warp CTAs give 28
    t = per_sm_table(64)
    assert busiest(4096, 8) == 32 and busiest(4096, 7) == 28
    assert rlib.rans_check_cta_warps(4096, SMS, t, 8) == 7


def test_rule_against_brute_force(rlib):
    """Over random occupancy tables and sizes: the chosen size fits in one
    wave, no fitting size gives the busiest SM fewer warps, and no larger
    fitting size gives it as few."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        W = int(rng.integers(1, 9))
        sms = int(rng.integers(1, 200))
        t = [0] + [int(v) for v in rng.integers(0, 33, size=W)]
        n = int(rng.integers(1, 3 * max(1, t[W]) * sms * W + 2))
        w = rlib.rans_check_cta_warps(n, sms, t, W)
        if t[W] <= 0 or n > t[W] * sms * W:
            assert w == W
            continue
        fits = [v for v in range(1, W + 1) if t[v] > 0 and -(-n // v) <= t[v] * sms]
        assert w in fits
        best = min(busiest(n, v, sms) for v in fits)
        assert busiest(n, w, sms) == best
        assert all(busiest(n, v, sms) > best for v in fits if v > w)


@pytest.mark.parametrize("n,sms,W", list(itertools.product([0, 1, 5], [0, 3], [1, 4])))
def test_degenerate_inputs(rlib, n, sms, W):
    t = [0] + [4] * W
    w = rlib.rans_check_cta_warps(n, sms, t, W)
    assert 1 <= w <= W
    if sms == 0:
        assert w == W


def test_bad_arguments(rlib):
    assert rlib.lib.rans_check_cta_warps(10, SMS, None, 8) == 0
    assert rlib.rans_check_cta_warps(10, SMS, [0] * 34, 33) == 0
