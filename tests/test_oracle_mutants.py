"""Each planted mistake in the oracle must be caught by at least one pin.

The mutants are compiled from the same source with -DORACLE_MUTANT=k:
  1 drops B_s from C            2 swaps M and f in C
  3 emits floor(x/b), not x mod b   4 assigns symbol i to coder (i+1) mod N
  5 leaves the words in emission order   6 starts the coders at L+1
  7 off-by-one symbol search in D        8 quantizer ties go to the higher index
  9 sends a symbol's raw (bypass) digits after encoding it, not before
 10 lays a width-baked step's digits out depth-first, not breadth-first
 11 updates an adaptive context before coding the symbol, not after
 12 muxes the coders' buffers by concatenation, not in the decoders' read order
 13 hands out canonical codes of one length in decreasing symbol order
 14 updates an adaptive n-symbol model before coding the symbol, not after
 15 moves the coded symbol's lower boundary up with the ones above it
"""
import pytest

import oracle
import oracle_pins

MUTANTS = range(1, 16)


@pytest.mark.parametrize("k", MUTANTS)
def test_mutant_is_caught(k):
    o = oracle.Oracle(mutant=k)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(o)
        except (AssertionError, oracle.OracleError, IndexError, ValueError, ZeroDivisionError):
            caught.append(pin.__name__)
    assert caught, f"mutant {k} passed every pin"
