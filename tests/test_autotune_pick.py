"""The autotuner's choice among timed candidates (host logic; no GPU)."""
from paper_2308_12698_b300.autotune import pick_step


def test_fastest_wins_outside_the_tie_band():
    # 128 is 2 % slower than 64: the fastest is taken
    assert pick_step([(10.00, 64, 1000), (10.20, 128, 1000), (10.30, 256, 1000)]) == (10.00, 64, 1000)


def test_ties_go_to_the_larger_block_then_the_larger_k():
    res = [(9.930, 32, 1000), (9.935, 64, 1000), (9.931, 128, 100), (9.933, 128, 1000), (10.10, 256, 1000)]
    assert pick_step(res) == (9.933, 128, 1000)


def test_tie_band_is_relative():
    assert pick_step([(100.0, 32, 10), (100.4, 256, 10)])[1] == 256
    assert pick_step([(100.0, 32, 10), (100.6, 256, 10)])[1] == 32
    assert pick_step([(100.0, 32, 10), (100.6, 256, 10)], tie=0.01)[1] == 256


def test_single_candidate():
    assert pick_step([(1.0, 128, 10)]) == (1.0, 128, 10)
