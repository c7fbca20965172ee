"""Host logic of the autotuner: coordinate descent over the plan knobs,
driven by synthetic cost functions (no GPU)."""
import dataclasses

from paper_1510_00844_gb300.autotune import SPACE, descend
from paper_1510_00844_gb300.spgemm import Tuning


def test_descent_finds_the_minimum_of_a_separable_cost():
    best_vals = {"dense_min_flops": 256, "hash_shift": 1, "dense_chunk": 2048, "seg_log2": 18}

    def cost(t: Tuning) -> float:
        c = 10.0
        for k, v in best_vals.items():
            c += 0.0 if getattr(t, k) == v else 1.0
        return c

    best, table = descend(cost, SPACE)
    assert all(getattr(best, k) == v for k, v in best_vals.items())
    assert len(table) == len(set(table))             # each candidate measured once
    assert Tuning() in table                         # the library default is the baseline


def test_descent_keeps_the_default_without_a_real_gain():
    best, table = descend(lambda t: 5.0 - 0.01 * t.hash_shift, SPACE, min_gain=0.02)
    assert best == Tuning()


def test_equal_settings_are_measured_once():
    calls = []
    best, table = descend(lambda t: calls.append(t) or 1.0, SPACE)
    # Tuning() and the spelled-out default dense_min_flops=1024 are one setting
    assert Tuning(dense_min_flops=1024) in table
    assert len(calls) == len(table) - 1


def test_descent_is_coordinate_wise():
    seen = []

    def cost(t: Tuning) -> float:
        seen.append(t)
        return 1.0 if t.dense_min_flops == 512 else 2.0

    best, table = descend(cost, {"dense_min_flops": (1024, 512), "hash_shift": (0, 1)})
    assert best.dense_min_flops == 512
    # later knobs are tried on top of the best value found so far
    assert dataclasses.replace(best, hash_shift=1) in table
    # the default and its spelled-out dense_min_flops=1024 are measured once
    assert len(table) == 4 and len(seen) == 3
