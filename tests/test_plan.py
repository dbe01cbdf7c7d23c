"""Host logic of the step schedule (seeds_plan, no GPU): every op of every
image runs once, in order, one op per step; a phase's moves are replayed
exactly once into the buffer it read (fused into the next phase of the same
level, or as a catch-up entry beside the next op); the fusion follows the
step's size; the virtual threads of a step are laid out without gaps."""
import ctypes

import pytest

from paper_1309_3848_gb300 import binding as b
from paper_1309_3848_gb300 import synth

INIT, PHASE, DESCEND, OUTPUT, CATCHUP, MINIT, MPHASE, BTILE = range(8)


def kind_of(e):
    """The op an entry runs: a block phase in warp tiles is a phase."""
    return PHASE if e["op"] == BTILE else e["op"]


def op_list(p):
    """The op list of an image (kind, level, phase), written out from the
    schedule the paper describes (Sec. 5: block levels L..1, then pixels;
    iterations of four parity phases per level) and the means iterations."""
    L, iters = p.block_levels, p.iters_per_level
    ops = [(INIT, 0, 0)]
    for level in range(L, -1, -1):
        for it in range(iters):
            for ph in range(4):
                ops.append((PHASE, level, ph))
        if level > 0:
            ops.append((DESCEND, level, 0))
    if p.means_iters > 0:
        ops.append((MINIT, 0, 0))
        for it in range(p.means_iters):
            for ph in range(4):
                ops.append((MPHASE, 0, ph))
    ops.append((OUTPUT, 0, 0))
    return ops


def padded(e):
    return (e["units"] * e["group"] + 31) // 32 * 32


def grid(p):
    rc, gx, gy = b.check_params(p)
    assert rc == 0
    L = p.block_levels
    return [(gx << (L - l + 1), gy << (L - l + 1)) if l > 0 else (p.width, p.height) for l in range(L + 1)]


def lattice(nx, ny, phase):
    px, py = phase & 1, phase >> 1
    return (nx - px + 1) >> 1, (ny - py + 1) >> 1


def params_of(job):
    L = min(job.levels, b.feasible_levels(job.image.width, job.image.height, job.num_superpixels))
    return b.make_params(job.image.width, job.image.height, job.num_superpixels, L, job.bins_per_channel,
                         job.iters_per_level, job.patch, job.gamma, job.color_space, job.means_iters,
                         job.compactness, job.edge_threshold)


CASES = {
    "1080p": [params_of(synth.plain_1080()[0])],
    "481": [params_of(synth.plain_481()[0])],
    "means": [b.make_params(200, 150, 60, 2, 5, 2, means_iters=2, compactness=10)],
    "L0": [b.make_params(64, 48, 12, 0, 5, 3)],
    "batch": [params_of(j) for j in synth.random_small_jobs(5, 12, max_side=300)],
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("sms", [1, 152, 1 << 20])
def test_every_op_runs_once_in_order_and_every_phase_is_replayed_once(case, sms):
    ps = CASES[case]
    steps = b.plan(ps, sms)
    ops = [op_list(p) for p in ps]
    assert len(steps) == max(len(o) for o in ops)
    seen = [[] for _ in ps]
    replayed = [set() for _ in ps]
    for s, (threads, ents) in enumerate(steps):
        for e in ents:
            i = e["img"]
            if e["op"] == CATCHUP:
                kind, level, phase = ops[i][e["opidx"] - 1]
                assert kind in (PHASE, MPHASE) and (e["level"], e["phase"]) == (level, phase)
                assert e["opidx"] == s
                replayed[i].add(e["opidx"] - 1)
                continue
            assert e["opidx"] == s, "image %d runs op %d at step %d" % (i, e["opidx"], s)
            assert (kind_of(e), e["level"]) == ops[i][s][:2]
            assert e["op"] != BTILE or e["level"] > 0
            if kind_of(e) in (PHASE, MPHASE):
                assert e["phase"] == ops[i][s][2]
            if e["cphase"] >= 0:  # fused: the previous op is a phase of the same kind and level
                kind, level, phase = ops[i][s - 1]
                assert (kind, level, phase) == (kind_of(e), e["level"], e["cphase"])
                replayed[i].add(s - 1)
            seen[i].append(s)
    for i, o in enumerate(ops):
        assert seen[i] == list(range(len(o)))
        # the output reads the buffer the last phase wrote its moves into:
        # that phase is not replayed
        phases = {s for s, (kind, _, _) in enumerate(o[:-2]) if kind in (PHASE, MPHASE)}
        assert o[-1][0] == OUTPUT and o[-2][0] in (PHASE, MPHASE)
        assert replayed[i] == phases, "phases never replayed: %s" % sorted(phases - replayed[i])


@pytest.mark.parametrize("case", sorted(CASES))
def test_virtual_threads_are_laid_out_without_gaps(case):
    for threads, ents in b.plan(CASES[case], 152):
        at = 0
        for e in ents:
            assert e["vt_begin"] == at and e["group"] in (1, 32) and e["units"] > 0
            at += padded(e)
        assert threads == at


def test_units_follow_the_lattices():
    p = CASES["1080p"][0]
    g = grid(p)
    for threads, ents in b.plan([p], 152):
        for e in ents:
            if e["op"] not in (PHASE, CATCHUP) or e["level"] == 0:
                continue
            nx, ny = g[e["level"]]
            cols, rows = lattice(nx, ny, e["phase"])
            if e["cphase"] >= 0:  # the union of both phases' lattices
                c2, r2 = lattice(nx, ny, e["cphase"])
                cols, rows = max(cols, c2), max(rows, r2)
            assert e["units"] == cols * rows  # 1080p has no wide step with 152 SMs
    # pixel phases: warp tiles of 32 x 4 (or 32 x 2) units; block phases of
    # warp-judged levels, in steps with at least two tiles per warp slot:
    # warp tiles of 32 x 1 units
    W, H = p.width, p.height

    def maxarea(level):
        nx, ny = g[level]
        w = max((i + 1) * W // nx - i * W // nx for i in range(nx))
        h = max((i + 1) * H // ny - i * H // ny for i in range(ny))
        return w * h

    for rows_per_tile in (4, 2):
        t = b.seeds_tuning(0, 0, 0, 16, rows_per_tile, 0)
        tiled = 0
        for threads, ents in b.plan([p], 1, t):  # one SM (32 warp slots): every step fused
            for e in ents:
                if e["op"] not in (PHASE, BTILE):
                    continue
                cols, rows = lattice(*g[e["level"]], e["phase"])
                if e["cphase"] >= 0:
                    c2, r2 = lattice(*g[e["level"]], e["cphase"])
                    cols, rows = max(cols, c2), max(rows, r2)
                if e["level"] == 0:
                    assert e["units"] == -(-cols // 32) * -(-rows // rows_per_tile) and e["group"] == 32
                    continue
                tiles = -(-cols // 32) * rows
                expect = maxarea(e["level"]) > 16 and tiles >= 2 * 32
                assert (e["op"] == BTILE) == expect, (e, tiles)
                if expect:
                    assert e["units"] == tiles and e["group"] == 32
                    tiled += 1
        # levels 4..2 of 1080p judge their blocks by warps; 2 and 3 have
        # more than 64 one-row tiles per phase
        assert tiled >= 2 * 4 * p.iters_per_level


def test_fusion_follows_the_step_size():
    """Below the machine's warp slots (sms x 32) block phases replay in
    catch-up entries; pixel phases only below an eighth of that."""
    p = CASES["1080p"][0]
    ops = op_list(p)
    for sms, fused in ((1, True), (1 << 20, False)):  # 32 warp slots; 33.5 M warp slots
        for threads, ents in b.plan([p], sms):
            for e in ents:
                if kind_of(e) == PHASE and ops[e["opidx"] - 1][:2] == (PHASE, e["level"]):
                    assert (e["cphase"] >= 0) == fused, (sms, e)
    # one 1080p image on 152 SMs (4,864 warp slots): level 4 (1,008 warps of
    # 484 px) and level 1 split, level 2 (16,128 warps) stays fused, and the
    # pixel phases (4,050 tiles, above 608) stay fused
    by_level = {}
    for threads, ents in b.plan([p], 152):
        for e in ents:
            if e["op"] == PHASE and e["phase"] != 0:
                by_level.setdefault(e["level"], set()).add(e["cphase"] >= 0)
    assert by_level == {4: {False}, 3: {False}, 2: {True}, 1: {False}, 0: {True}}
    # the 481x321 image's pixel phases (302 tiles) are below 608: split
    small = CASES["481"][0]
    pix = {e["cphase"] >= 0 for _, ents in b.plan([small], 152) for e in ents
           if e["op"] == PHASE and e["level"] == 0 and e["phase"] != 0}
    assert pix == {False}


def test_small_blocks_take_a_thread_each():
    p = CASES["481"][0]
    g = grid(p)
    W, H = p.width, p.height

    def maxarea(level):
        nx, ny = g[level]
        w = max((i + 1) * W // nx - i * W // nx for i in range(nx))
        h = max((i + 1) * H // ny - i * H // ny for i in range(ny))
        return w * h

    for area in (1, 4, 9, 16):
        t = b.seeds_tuning(0, 0, 0, area, 4)
        for _, ents in b.plan([p], 152, t):
            for e in ents:
                if e["op"] == PHASE and e["level"] > 0:
                    assert e["group"] == (1 if maxarea(e["level"]) <= area else 32)
                elif e["op"] == CATCHUP and e["level"] > 0:  # the 481x321 image has no wide step
                    assert e["group"] == (1 if maxarea(e["level"]) <= area else 32)


def test_catchup_entries_are_wide_only_in_wide_steps():
    """A catch-up gives a lane four pixels, a small block a lane each and a
    block a warp judges a warp each; in a wide step (block_tiles = 2: every
    step) a lane takes four small blocks, and blocks a warp judges of at
    most 128 pixels a lane each (the warp replays their moves)."""
    ps = [params_of(j) for j in synth.batch_4k(2)]
    g = grid(ps[0])
    W, H = ps[0].width, ps[0].height

    def maxarea(level):
        nx, ny = g[level]
        w = max((i + 1) * W // nx - i * W // nx for i in range(nx))
        h = max((i + 1) * H // ny - i * H // ny for i in range(ny))
        return w * h

    for policy in (1, 2):
        seen = set()
        for sms in (1 << 12, 1 << 16):  # many SMs: block replays in catch-up entries
            for _, ents in b.plan(ps, sms, b.seeds_tuning(0, 0, 0, 16, 4, policy)):
                for e in ents:
                    if e["op"] != CATCHUP:
                        continue
                    cols, rows = lattice(*g[e["level"]], e["phase"])
                    pu = cols * rows
                    area = maxarea(e["level"]) if e["level"] else 1
                    if e["level"] == 0:
                        want = (1, -(-pu // 4))
                    elif area > 16:
                        want = (32, pu) if policy == 1 or area > 128 else (1, pu)
                    else:
                        want = (1, pu) if policy == 1 else (1, -(-pu // 4))
                    assert (e["group"], e["units"]) == want, (policy, e, pu, area)
                    seen.add((e["level"], want[0], want[1] != pu))
        if policy == 1:
            assert {(1, 1, False), (2, 1, False), (3, 32, False), (4, 32, False), (5, 32, False)} <= seen, seen
        else:
            assert {(1, 1, True), (2, 1, True), (3, 1, False), (4, 1, False), (5, 32, False)} <= seen, seen


def test_block_steps_run_in_tiles_when_they_fill_the_machine_twice():
    """By default (block_tiles = 0) a step of warp-judged blocks runs in warp
    tiles of 32 x 1 units exactly when its tiles (fused form) number at least
    twice the machine's warp slots (sms x 32); otherwise, and always with
    block_tiles = 1, its blocks keep a warp each.  Blocks judged by a thread
    never run in tiles, and block_tiles = 2 tiles every warp-judged step."""
    ps = [params_of(j) for j in synth.batch_4k(4)]
    g = grid(ps[0])
    rule = b.seeds_tuning(0, 0, 0, 16, 4, 0)
    seen = set()
    for sms in (1, 16, 152, 1 << 12):
        for threads, ents in b.plan(ps, sms, rule):
            blocks = [e for e in ents if kind_of(e) == PHASE and e["level"] > 0]
            if not blocks:
                continue
            level, phase = blocks[0]["level"], blocks[0]["phase"]
            cols, rows = lattice(*g[level], phase)
            prev = [e["cphase"] for e in blocks if e["cphase"] >= 0]
            if prev:
                c2, r2 = lattice(*g[level], prev[0])
                cols, rows = max(cols, c2), max(rows, r2)
            warp = all(e["group"] == 32 for e in blocks)
            tiles = len(ps) * -(-cols // 32) * rows
            tiled = warp and tiles >= 2 * sms * 32
            seen.add((warp, tiled))
            assert all((e["op"] == BTILE) == tiled for e in blocks), (sms, level, tiles)
        never = b.seeds_tuning(0, 0, 0, 16, 4, 1)
        assert not any(e["op"] == BTILE for _, ents in b.plan(ps, sms, never) for e in ents)
        always = b.seeds_tuning(0, 0, 0, 16, 4, 2)
        for _, ents in b.plan(ps, sms, always):
            for e in ents:
                if kind_of(e) == PHASE and e["level"] > 0:
                    assert (e["op"] == BTILE) == (e["group"] == 32), (sms, e)
    assert seen == {(False, False), (True, False), (True, True)}


def test_small_block_warps_take_2d_blocks_where_superpixels_are_wide():
    """A small-block phase gives each warp 32 units of a row, or, on a level
    whose superpixels span at least 16 lattice units per side (2^(L - level):
    level 1 of L = 5), a block of 8 x 4 units; its entry then counts
    ceil(cols/8) * ceil(rows/4) warps."""
    for jobs, L2d in ((synth.batch_4k(2), {1}), (synth.plain_1080(), set())):
        ps = [params_of(j) for j in jobs]
        g = grid(ps[0])
        L = ps[0].block_levels
        seen = set()
        for sms in (1, 152):
            for threads, ents in b.plan(ps, sms):
                ends = [e["vt_begin"] for e in ents[1:]] + [threads]
                for e, end in zip(ents, ends):
                    if e["op"] != PHASE or e["level"] == 0 or e["group"] != 1:
                        continue
                    cols, rows = lattice(*g[e["level"]], e["phase"])
                    if e["cphase"] >= 0:
                        c2, r2 = lattice(*g[e["level"]], e["cphase"])
                        cols, rows = max(cols, c2), max(rows, r2)
                    assert e["units"] == cols * rows
                    if (1 << (L - e["level"])) >= 16:
                        want = -(-cols // 8) * -(-rows // 4) * 32
                    else:
                        want = -(-cols * rows // 32) * 32
                    assert end - e["vt_begin"] == want, (e, want)
                    seen.add(e["level"] if (1 << (L - e["level"])) >= 16 else -e["level"])
        assert {l for l in seen if l > 0} == L2d


def test_a_batch_shares_every_step():
    ps = CASES["batch"]
    steps = b.plan(ps, 152)
    for s, (_, ents) in enumerate(steps):
        imgs = {e["img"] for e in ents if e["op"] != CATCHUP}
        assert imgs == {i for i, p in enumerate(ps) if len(op_list(p)) > s}


def test_bad_inputs():
    p = CASES["481"][0]
    arr = (b.seeds_params * 1)(p)
    ne, ns = ctypes.c_int32(), ctypes.c_int32()

    def call(params, n, tuning, sms, ob=None, oe=None, out=None, cap=0, first=None, step_cap=0):
        return b.lib.seeds_plan(params, n, tuning, sms, ob, oe, out, cap, ctypes.byref(ne), first, None, step_cap,
                                ctypes.byref(ns))

    assert call(arr, 0, None, 152) == b.SEEDS_ERR_INVALID
    assert call(arr, 1, None, 0) == b.SEEDS_ERR_INVALID
    assert call(arr, 1, None, 152) == 0
    small = (b.seeds_plan_entry * 1)()
    first = (ctypes.c_int32 * 2)()
    assert call(arr, 1, None, 152, out=small, cap=1, first=first, step_cap=2) == b.SEEDS_ERR_INVALID
    bad_tuning = b.seeds_tuning(0, 0, 0, 17, 4)
    assert call(arr, 1, ctypes.byref(bad_tuning), 152) == b.SEEDS_ERR_INVALID
    nops = len(op_list(p))
    for ob, oe in ((-1, 3), (5, 4), (0, nops + 1)):
        assert call(arr, 1, None, 152, (ctypes.c_int32 * 1)(ob), (ctypes.c_int32 * 1)(oe)) == b.SEEDS_ERR_INVALID
    geo = (b.seeds_params * 1)(b.make_params(16, 16, 4, 4, 5, 1))
    assert call(geo, 1, None, 152) == b.SEEDS_ERR_GEOMETRY


@pytest.mark.parametrize("case", ["1080p", "means", "batch"])
def test_a_run_split_into_launches_runs_every_op_once(case):
    """Launches that stop at chosen ops and resume there (anytime stops,
    op ranges) together run every op once, in order, and replay every phase
    once: a launch that starts after a phase catches its moves up first."""
    ps = CASES[case]
    ops = [op_list(p) for p in ps]
    cuts = sorted({0, 1, 5, 17, 40, 41, 60, max(len(o) for o in ops)})
    seen = [[] for _ in ps]
    replayed = [set() for _ in ps]
    for lo, hi in zip(cuts, cuts[1:]):
        ob = [min(lo, len(o)) for o in ops]
        oe = [min(hi, len(o)) for o in ops]
        for s, (_, ents) in enumerate(b.plan(ps, 152, op_begin=ob, op_end=oe)):
            for e in ents:
                i = e["img"]
                if e["op"] == CATCHUP:
                    replayed[i].add(e["opidx"] - 1)
                    continue
                assert e["opidx"] == ob[i] + s
                if e["cphase"] >= 0:
                    replayed[i].add(e["opidx"] - 1)
                seen[i].append(e["opidx"])
    for i, o in enumerate(ops):
        assert seen[i] == list(range(len(o)))
        assert replayed[i] == {s for s, (kind, _, _) in enumerate(o[:-2]) if kind in (PHASE, MPHASE)}
