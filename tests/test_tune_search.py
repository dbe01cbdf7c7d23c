"""The autotuner's search (seeds_tune_search, the code seeds_autotune runs)
with synthetic timings on the host: one pass of coordinate descent over the
six launch knobs in a fixed order, a 2% bar for a change, settings that
cannot run never chosen, every candidate timed once."""
import math

from paper_1309_3848_gb300 import binding as b

KNOBS = [("threads_per_block", (128, 256, 512, 1024)), ("blocks_per_sm", (0, 1, 2, 3)), ("hist_layout", (0, 1)),
         ("small_block_area", (4, 9, 16)), ("pixel_tile_rows", (2, 4)), ("block_tiles", (0, 1, 2))]
START = (1024, 0, 0, 16, 4, 0)


def key(t):
    return tuple(getattr(t, k) for k, _ in KNOBS)


def run(cost, start=START):
    calls = []

    def timed(t):
        calls.append(key(t))
        return cost(dict(zip([k for k, _ in KNOBS], key(t))))

    best = b.tune_search(b.seeds_tuning(*start), timed)
    return key(best), calls


def test_separable_costs_reach_the_minimum_of_every_knob():
    want = {"threads_per_block": 256, "blocks_per_sm": 2, "hist_layout": 1, "small_block_area": 4,
            "pixel_tile_rows": 2, "block_tiles": 1}
    best, calls = run(lambda t: 1.0 + sum(0.1 * (t[k] != v) for k, v in want.items()))
    assert best == tuple(want[k] for k, _ in KNOBS)
    # the start, then each knob's values other than the current one as the
    # pass reaches them; every value of every knob is timed
    assert 1 + sum(len(vals) - 1 for _, vals in KNOBS) <= len(calls) <= 1 + sum(len(vals) for _, vals in KNOBS)
    for knob, (_, vals) in enumerate(KNOBS):
        assert {c[knob] for c in calls} >= set(vals)


def test_a_change_must_win_by_two_percent():
    # 1% faster threads, 3% faster tile rows: only the tile rows move
    best, _ = run(lambda t: 1.0 - 0.01 * (t["threads_per_block"] == 512) - 0.03 * (t["pixel_tile_rows"] == 2))
    assert best == (1024, 0, 0, 16, 2, 0)


def test_settings_that_cannot_run_are_never_taken():
    best, _ = run(lambda t: math.inf if t["threads_per_block"] == 1024 and t["blocks_per_sm"] == 0 else 2.0)
    # the start itself cannot run: the first value that can replaces it
    assert best[0] != 1024 or best[1] != 0
    best, _ = run(lambda t: math.inf if t["hist_layout"] == 1 else 1.0 + 0.5 * (t["small_block_area"] != 9))
    assert best[2] == 0 and best[3] == 9


def test_one_pass_in_knob_order():
    # each knob is set while the earlier knobs' choices stand: the threads
    # knob is chosen under blocks_per_sm = 0, so a better pair found only
    # with blocks_per_sm = 1 is not reached
    def cost(t):
        if t["threads_per_block"] == 128 and t["blocks_per_sm"] == 1:
            return 0.5
        return 1.0 - 0.1 * (t["blocks_per_sm"] == 1)

    best, calls = run(cost)
    assert best[:2] == (1024, 1)
    first_of = {}
    for i, c in enumerate(calls[1:]):
        for knob, v in enumerate(c):
            if v != START[knob] and knob not in first_of:
                first_of[knob] = i
    assert [first_of[k] for k in sorted(first_of)] == sorted(first_of.values())
