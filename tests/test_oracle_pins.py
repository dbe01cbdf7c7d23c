"""Pins for the oracle: what the paper and the mathematics fix, checked
against the oracle's C code without trusting any of its formulas.

Covered: the colour bins (equal-width intervals, R-major order), the grid
geometry (closed-form counts, nesting, non-empty blocks), the initial grid
and its histograms, per-phase invariants (histograms equal a recount, one
label per pixel, every label present and 4-connected, block homogeneity),
every decision of every phase against a brute-force restatement in exact
fractions, Prop. 2 as an exact identity, the block test at |L| = 1 against the
single-lookup pixel test, special cases with known answers, and the
sequential mode's energy ascent.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import brute
from oracle import energy, ref
from paper_1309_3848_gb300 import synth


def rgb_noise(W, H, seed, lo=0, hi=256):
    return np.random.default_rng(seed).integers(lo, hi, size=(H, W, 3)).astype(np.uint8)


def recount(labels, bins, K, nbins):
    h = np.zeros((K, nbins), np.int64)
    np.add.at(h, (labels.ravel(), bins.ravel()), 1)
    return h, np.bincount(labels.ravel(), minlength=K).astype(np.int64)


def four_connected(mask):
    """Number of 4-connected components of a boolean mask (plain BFS)."""
    H, W = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    comps = 0
    for y0, x0 in zip(*np.nonzero(mask)):
        if seen[y0, x0]:
            continue
        comps += 1
        stack = [(y0, x0)]
        seen[y0, x0] = True
        while stack:
            y, x = stack.pop()
            for ny, nx in ((y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)):
                if 0 <= ny < H and 0 <= nx < W and mask[ny, nx] and not seen[ny, nx]:
                    seen[ny, nx] = True
                    stack.append((ny, nx))
    return comps


def assert_valid_partition(labels, K):
    assert labels.min() >= 0 and labels.max() < K
    present = np.unique(labels)
    assert len(present) == K, "a superpixel vanished"
    for k in range(K):
        assert four_connected(labels == k) == 1, "superpixel %d is split" % k


# --------------------------------------------------------------------------
# colour bins (R1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("B", list(range(1, 17)))
def test_bins_are_equal_width_and_r_major(B):
    v = np.arange(256, dtype=np.uint8)
    # one row per channel under test; the other two channels held at 0
    img = np.zeros((3, 256, 3), np.uint8)
    for c in range(3):
        img[c, :, c] = v
    r = ref.Ref(256, 3, 1, 0, B, 1)
    r.init(img)
    bins = r.bins()
    per_channel = [bins[0] // (B * B), (bins[1] // B) % B, bins[2] % B]
    weights = [B * B, B, 1]
    for c in range(3):
        b = per_channel[c]
        # only this channel's digit moves, in place value B^2, B, 1
        assert np.array_equal(bins[c], b * weights[c])
        assert b[0] == 0 and b[-1] == B - 1
        assert np.all(np.diff(b) >= 0) and np.all(np.diff(b) <= 1)
        widths = np.bincount(b, minlength=B)
        assert set(widths.tolist()) <= {256 // B, -(-256 // B)}
        # bin b covers [b*256/B, (b+1)*256/B): the lowest member is ceil(b*256/B)
        starts = [int(np.argmax(b == t)) for t in range(B)]
        assert starts == [-(-t * 256 // B) for t in range(B)]
    assert r.nbins == B ** 3


# --------------------------------------------------------------------------
# geometry (R3)
# --------------------------------------------------------------------------

def test_superpixel_counts_of_the_workloads():
    # gx = round(sqrt(K W/H)), gy = round(K/gx)
    assert ref.grid(481, 321, 200, 4)[1:] == (17, 12)
    assert ref.grid(1920, 1080, 1000, 4)[1:] == (42, 24)
    assert ref.grid(3840, 2160, 5000, 5)[1:] == (94, 53)
    assert ref.grid(320, 240, 1500, 2) == (0, 45, 33)
    assert ref.grid(320, 240, 1500, 3)[0] == ref.EGEOM  # 45*8 > 320


@pytest.mark.parametrize("W,H,K,L", [(481, 321, 200, 4), (64, 48, 12, 3), (33, 17, 5, 2), (1920, 1080, 1000, 4),
                                     (20, 20, 1, 4), (7, 5, 35, 0)])
def test_levels_nest_and_blocks_are_non_empty(W, H, K, L):
    r = ref.Ref(W, H, K, L, 5, 1)
    sx = [(i * W) // r.gx for i in range(r.gx + 1)]
    sy = [(i * H) // r.gy for i in range(r.gy + 1)]
    prev = None
    for level in range(L, -1, -1):
        nbx, nby, xe, ye = r.level_grid(level)
        assert xe[0] == 0 and xe[-1] == W and ye[0] == 0 and ye[-1] == H
        assert np.all(np.diff(xe) >= 1) and np.all(np.diff(ye) >= 1)
        if level == L and L > 0:
            # level L: a superpixel is exactly 2x2 blocks
            assert nbx == 2 * r.gx and nby == 2 * r.gy
            assert list(xe[::2]) == sx and list(ye[::2]) == sy
        if prev is not None and level > 0:
            # every edge of the coarser level is an edge of this one (2x2 joining)
            assert set(prev[0].tolist()) <= set(xe.tolist()) and nbx == 2 * (len(prev[0]) - 1)
            assert set(prev[1].tolist()) <= set(ye.tolist()) and nby == 2 * (len(prev[1]) - 1)
        if level == 0:
            assert nbx == W and nby == H
        prev = (xe, ye)


def test_smallest_blocks_are_small():
    # the paper's smallest blocks are 2x2 or 3x3 pixels (Sec. 5.1)
    for (W, H, K, L) in [(481, 321, 200, 4), (1920, 1080, 1000, 4), (3840, 2160, 5000, 5)]:
        r = ref.Ref(W, H, K, L, 5, 1)
        _, _, xe, ye = r.level_grid(1)
        assert np.diff(xe).max() <= 3 and np.diff(ye).max() <= 3


def test_invalid_parameters_are_rejected():
    with pytest.raises(ref.OracleError):
        ref.Ref(0, 5, 1, 0, 5, 1)
    with pytest.raises(ref.OracleError):
        ref.Ref(16, 16, 4, 0, 17, 1)
    with pytest.raises(ref.OracleError):
        ref.Ref(16, 16, 4, 0, 5, 1, patch=5)
    with pytest.raises(ref.OracleError) as e:
        ref.Ref(16, 16, 4, 4, 5, 1)  # 2 * 2^4 > 16
    assert e.value.code == ref.EGEOM


# --------------------------------------------------------------------------
# initial grid and histograms (Sec. 5.1, Eq. 4)
# --------------------------------------------------------------------------

def test_initial_partition_is_the_grid():
    W, H, K = 53, 37, 12
    r = ref.Ref(W, H, K, 2, 4, 1)
    img = rgb_noise(W, H, 1)
    r.init(img)
    lab = r.labels()
    sx = [(i * W) // r.gx for i in range(r.gx + 1)]
    sy = [(i * H) // r.gy for i in range(r.gy + 1)]
    for y in range(H):
        for x in range(W):
            cx = max(i for i in range(r.gx) if sx[i] <= x)
            cy = max(i for i in range(r.gy) if sy[i] <= y)
            assert lab[y, x] == cy * r.gx + cx
    h, s = r.hist()
    h2, s2 = recount(lab, r.bins(), r.K, r.nbins)
    assert np.array_equal(h, h2) and np.array_equal(s, s2)


# --------------------------------------------------------------------------
# invariants after every phase
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_invariants_after_every_phase(seed):
    jobs = synth.random_small_jobs(100 + seed, 1, max_side=40)
    job = jobs[0]
    W, H = job.image.width, job.image.height
    L = job.levels
    while L > 0 and ref.grid(W, H, job.num_superpixels, L)[0] != 0:
        L -= 1
    r = ref.Ref(W, H, job.num_superpixels, L, job.bins_per_channel, job.iters_per_level, job.patch, job.gamma)
    img = synth.make_image(job.image)
    r.init(img)
    bins = r.bins()
    last_level = None
    for level, phase in r.schedule():
        if level != last_level:
            # at the start of a level every unit carries one label
            nbx, nby, xe, ye = r.level_grid(level)
            lab = r.labels()
            for by in range(nby):
                for bx in range(nbx):
                    blk = lab[ye[by]:ye[by + 1], xe[bx]:xe[bx + 1]]
                    assert np.all(blk == blk[0, 0])
            last_level = level
        r.run_phase(level, phase)
        lab = r.labels()
        h, s = r.hist()
        h2, s2 = recount(lab, bins, r.K, r.nbins)
        assert np.array_equal(h, h2) and np.array_equal(s, s2)
        assert_valid_partition(lab, r.K)


# --------------------------------------------------------------------------
# every decision against the brute-force restatement (exact fractions)
# --------------------------------------------------------------------------

BRUTE_CASES = [
    # W, H, K, L, B, iters, patch, gamma, image seed
    (16, 16, 4, 2, 3, 2, 3, (1, 1), 1),
    (17, 13, 6, 1, 4, 2, 3, (1, 1), 2),
    (20, 14, 5, 2, 2, 1, 0, (1, 1), 3),
    (15, 15, 9, 1, 5, 2, 3, (3, 2), 4),
    (24, 10, 4, 2, 3, 1, 3, (0, 1), 5),
    (12, 18, 6, 0, 4, 3, 3, (2, 1), 6),
]


@pytest.mark.parametrize("case", BRUTE_CASES)
def test_every_decision_matches_brute_force(case):
    W, H, K, L, B, iters, patch, gamma, seed = case
    r = ref.Ref(W, H, K, L, B, iters, patch, gamma)
    # piecewise-constant colours plus noise, so moves actually happen
    spec = synth.ImageSpec(W, H, seed=seed, cells=5, sigma=20.0)
    img = synth.make_image(spec)
    r.init(img)
    bins = r.bins()
    total = 0
    for level, phase in r.schedule():
        _, _, xe, ye = r.level_grid(level)
        before = r.labels()
        dec = brute.phase_decisions(before, bins, r.nbins, level, phase, xe, ye, gamma, patch)
        n = r.run_phase(level, phase)
        assert n == len(dec)
        assert np.array_equal(r.labels(), brute.apply_decisions(before, dec, xe, ye))
        total += n
    assert total > 0


# --------------------------------------------------------------------------
# Prop. 2 as an exact identity (App. A.2)
# --------------------------------------------------------------------------

def test_prop2_identity_on_random_labelings():
    rng = np.random.default_rng(7)
    for trial in range(12):
        W, H = int(rng.integers(3, 9)), int(rng.integers(3, 9))
        K = int(rng.integers(2, 5))
        # any labeling works for the identity, connected or not
        labels = rng.integers(0, K, size=(H, W)).astype(np.int32)
        if ref.grid(W, H, K)[0] != 0:
            continue
        rK = ref.Ref(W, H, K, 0, 1, 1)
        if rK.K != K:
            continue
        rK.init(np.zeros((H, W, 3), np.uint8))
        rK.set_labels(labels)
        for y, x in itertools.product(range(H), range(W)):
            k = int(labels[y, x])
            for n in range(K):
                if n == k:
                    continue
                Gk, Kp = rK.patch_label_count(x, y, k)
                Gn, _ = rK.patch_label_count(x, y, n)
                before = energy.boundary_term_counts(labels)
                moved = labels.copy()
                moved[y, x] = n
                after = energy.boundary_term_counts(moved)
                # Z^2 (G(s) - G(s_t)) = 2 (G_n + |K_p| - G_k)
                assert after - before == 2 * (Gn + Kp - Gk)
                # |K_p| = in-image pixels of the 3x3 around p
                assert Kp == (min(x + 1, W - 1) - max(x - 1, 0) + 1) * (min(y + 1, H - 1) - max(y - 1, 0) + 1)


# --------------------------------------------------------------------------
# block test at |L| = 1 equals the single-lookup pixel test (Sec. 5)
# --------------------------------------------------------------------------

def test_one_pixel_blocks_decide_like_pixels():
    # W = gx * 2^L makes every level-1 block a single pixel
    W = H = 16
    for seed in range(3):
        r = ref.Ref(W, H, 4, 3, 3, 1, patch=0)
        assert (r.gx, r.gy) == (2, 2)
        nbx, nby, xe, ye = r.level_grid(1)
        assert (nbx, nby) == (W, H) and list(xe) == list(range(W + 1))
        r.init(synth.make_image(synth.ImageSpec(W, H, seed=seed, cells=4, sigma=25.0)))
        checked = 0
        for level, phase in r.schedule():
            if level == 1:
                for y in range(H):
                    for x in range(W):
                        assert r.decide(1, x, y) == r.decide(0, x, y)
                        checked += r.decide(0, x, y) >= 0
            r.run_phase(level, phase)
        assert checked > 0


# --------------------------------------------------------------------------
# special cases with known answers
# --------------------------------------------------------------------------

def grid_labels(r):
    W, H = r.W, r.H
    sx = np.array([(i * W) // r.gx for i in range(r.gx + 1)])
    sy = np.array([(i * H) // r.gy for i in range(r.gy + 1)])
    cx = np.searchsorted(sx, np.arange(W), side="right") - 1
    cy = np.searchsorted(sy, np.arange(H), side="right") - 1
    return (cy[:, None] * r.gx + cx[None, :]).astype(np.int32)


@pytest.mark.parametrize("gamma", [(0, 1), (1, 1), (5, 1)])
@pytest.mark.parametrize("B", [1, 5])
def test_constant_image_keeps_the_grid(gamma, B):
    r = ref.Ref(48, 40, 12, 2, B, 2, 3, gamma)
    img = np.full((40, 48, 3), 97, np.uint8)
    assert np.array_equal(r.run(img), grid_labels(r))


def test_one_bin_without_boundary_term_keeps_the_grid():
    r = ref.Ref(40, 32, 8, 2, 1, 2, 3, (0, 1))
    assert np.array_equal(r.run(rgb_noise(40, 32, 3)), grid_labels(r))


def test_grid_aligned_colour_edge_keeps_the_grid():
    # two flat colours split along a superpixel column edge
    r = ref.Ref(64, 32, 8, 2, 5, 2)
    img = np.zeros((32, 64, 3), np.uint8)
    img[:, :32] = (200, 30, 30)
    img[:, 32:] = (20, 20, 220)
    assert (r.gx, r.gy) == (4, 2)
    assert np.array_equal(r.run(img), grid_labels(r))


def test_boundaries_snap_to_an_off_grid_colour_edge():
    # colour edge at x = 37 inside the superpixel column [32, 48)
    r = ref.Ref(64, 32, 8, 2, 5, 3)
    img = np.zeros((32, 64, 3), np.uint8)
    img[:, :37] = (200, 30, 30)
    img[:, 37:] = (20, 20, 220)
    lab = r.run(img)
    # every pair of horizontally adjacent pixels across the colour edge
    # now belongs to two different superpixels
    assert np.all(lab[:, 36] != lab[:, 37])
    # and no superpixel spans both colours
    for k in range(r.K):
        xs = np.nonzero(lab == k)[1]
        assert xs.max() < 37 or xs.min() >= 37


# --------------------------------------------------------------------------
# sequential mode (the paper's order): energy ascent
# --------------------------------------------------------------------------

def unit_pixels(r, level, unit):
    nbx, nby, xe, ye = r.level_grid(level)
    bx, by = unit % nbx, unit // nbx
    return slice(ye[by], ye[by + 1]), slice(xe[bx], xe[bx + 1])


# In the literal energy G outweighs H by about |A| (a pixel move changes G by
# ~18/81 but H by ~1/|A|), so gamma is kept small here to leave both active.
@pytest.mark.parametrize("seed,gamma,patch", [(1, (1, 32), 3), (2, (0, 1), 3), (3, (1, 64), 3), (4, (1, 1), 0)])
def test_exact_sequential_mode_raises_energy_on_every_move(seed, gamma, patch):
    W, H = 24, 20
    r = ref.Ref(W, H, 6, 2, 3, 2, patch, gamma)
    img = synth.make_image(synth.ImageSpec(W, H, seed=seed, cells=5, sigma=18.0))
    final, trace, n = r.sequential(img, seed=seed, exact=True)
    assert n == len(trace) and n > 0
    bins = r.bins()
    lab = grid_labels(r)
    g = Fraction(*gamma)
    E = energy.energy(lab, bins, g, patch)
    for level, unit, k, nlab in trace.tolist():
        sl = unit_pixels(r, level, unit)
        assert np.all(lab[sl] == k)
        lab[sl] = nlab
        E2 = energy.energy(lab, bins, g, patch)
        assert E2 > E
        E = E2
    assert np.array_equal(lab, final)
    assert_valid_partition(final, r.K)


def test_proxy_sequential_with_one_bin_climbs_the_boundary_term():
    # with one colour bin the colour test always ties, so every accepted move
    # is a pure Prop. 2 decision, which is exact: G rises on each of them
    W, H = 24, 24
    r = ref.Ref(W, H, 9, 2, 1, 2, 3, (1, 1))
    img = rgb_noise(W, H, 9)
    # start from a ragged partition so that the boundary term has work to do
    final, trace, n = r.sequential(img, seed=5, exact=False)
    lab = grid_labels(r)
    G = energy.boundary_term_counts(lab)
    for level, unit, k, nlab in trace.tolist():
        sl = unit_pixels(r, level, unit)
        lab[sl] = nlab
        G2 = energy.boundary_term_counts(lab)
        assert G2 > G
        G = G2
    assert np.array_equal(lab, final)


def test_sequential_draws_are_the_published_splitmix64_outputs():
    """R14's generator against the published outputs of SplitMix64 from
    state 0 (tests/golden/splitmix64_state0.txt)."""
    want = [int(l.split()[0], 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and l[0] != "#"]
    assert len(want) == 5 and ref.splitmix64_draws(0, len(want)) == want


def test_sequential_visiting_order_is_a_uniform_permutation():
    """R14 visits the units of a sweep in a uniformly random order: over
    many seeds every one of the n! orders of n units occurs, at frequencies
    a chi-square test accepts (Sattolo's variant, a draw below u instead of
    up to u, makes only the cyclic orders; a skipped swap or a biased index
    leaves orders out or skews them)."""
    trials = 24000
    for n in (1, 2, 3, 4):
        counts = {}
        for seed in range(trials):
            o = tuple(ref.unit_order(seed, n).tolist())
            counts[o] = counts.get(o, 0) + 1
        assert set(counts) == set(itertools.permutations(range(n))), n
        fact = len(counts)
        e = trials / fact
        chi2 = sum((c - e) ** 2 / e for c in counts.values())
        # upper 0.01% points of chi-square with fact-1 = 0, 1, 5, 23 degrees of freedom
        assert chi2 <= {1: 0.0, 2: 15.2, 6: 25.8, 24: 57.1}[fact], (n, chi2)


def test_sequential_candidate_pick_is_uniform():
    """R14's proposal: one of a unit's nc candidates, each equally likely
    (chi-square over 60,000 picks), taken from the generator's draws."""
    want = [int(l.split()[0], 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and l[0] != "#"]
    for nc in (1, 2, 3, 4):
        picks = ref.candidate_picks(0, nc, 60000)
        assert [int(v) for v in picks[:5]] == [w % nc for w in want]
        counts = np.bincount(picks, minlength=nc)
        assert len(counts) == nc and counts.min() > 0
        e = len(picks) / nc
        chi2 = float(((counts - e) ** 2 / e).sum())
        # upper 0.01% points of chi-square with nc-1 = 0..3 degrees of freedom
        assert chi2 <= {1: 0.0, 2: 15.2, 3: 18.5, 4: 21.2}[nc], (nc, chi2)


def test_prop1_agreement_rate_is_high():
    """Diagnostic for Prop. 1 (an approximation; the paper reports agreement
    of 89-97%): over the parity schedule's pixel moves on a few noisy
    images, how often does an accepted move raise the exact colour term H?
    Loose band only: the test images are far smaller than the paper's."""
    agree = total = 0
    for (W, H, K, B, seed, cells, sigma) in [(32, 24, 8, 4, 11, 6, 15.0), (48, 48, 6, 5, 11, 6, 10.0),
                                             (48, 48, 6, 5, 12, 8, 6.0), (64, 48, 6, 5, 13, 6, 8.0)]:
        r = ref.Ref(W, H, K, 2, B, 2, 0)
        r.init(synth.make_image(synth.ImageSpec(W, H, seed=seed, cells=cells, sigma=sigma)))
        bins = r.bins()
        for level, phase in r.schedule():
            before = r.labels()
            r.run_phase(level, phase)
            after = r.labels()
            if level != 0:
                continue
            H0 = energy.colour_term(before, bins)
            for y, x in zip(*np.nonzero(before != after)):
                moved = before.copy()
                moved[y, x] = after[y, x]
                total += 1
                agree += energy.colour_term(moved, bins) > H0
    print("Prop. 1 agreement on accepted pixel moves: %d / %d" % (agree, total))
    assert total > 500
    assert agree / total >= 0.8, (agree, total)


# --------------------------------------------------------------------------
# constructed configurations: candidate ties and the ring rule
# --------------------------------------------------------------------------

RED, BLUE, GREEN = (220, 20, 20), (20, 20, 220), (20, 220, 20)


def constructed_state(labels, blue_labels, p):
    """16x16 state with 1-pixel level-1 blocks (gx = gy = 2, L = 3): pixels of
    `blue_labels` and the pixel p are blue, label 0 is red, the rest green."""
    img = np.zeros((16, 16, 3), np.uint8)
    img[:] = GREEN
    img[labels == 0] = RED
    for b in blue_labels:
        img[labels == b] = BLUE
    img[p[1], p[0]] = BLUE
    r = ref.Ref(16, 16, 4, 3, 5, 1, patch=0)
    r.init(img)
    r.set_labels(labels)
    return r


def t_junction(left, right):
    """p = (6,6) in label 0 (a red row above), `left` and `right` on its
    sides, `left` below: one run of 0 in the ring, so p may leave 0."""
    lab = np.full((16, 16), 3, np.int32)
    x0, y0 = 6, 6
    lab[y0 - 1, x0 - 2:x0 + 3] = 0
    lab[y0, x0 - 2:x0] = left
    lab[y0, x0] = 0
    lab[y0, x0 + 1:x0 + 3] = right
    lab[y0 + 1, x0 - 2:x0 + 1] = left
    lab[y0 + 1, x0 + 1:x0 + 3] = right
    return lab, (x0, y0)


@pytest.mark.parametrize("left,right", [(1, 2), (2, 1)])
def test_equal_candidates_go_to_the_smallest_label(left, right):
    lab, p = t_junction(left, right)
    r = constructed_state(lab, [1, 2], p)
    # both neighbours are all blue like p: f(1) == f(2) > f_stay = 0
    assert r.decide(0, *p) == 1
    assert r.decide(1, *p) == 1


def test_isolated_diagonal_cell_does_not_block_a_move():
    lab = np.full((16, 16), 3, np.int32)
    x0, y0 = 6, 6
    lab[:y0 + 1, x0] = 0            # label 0 comes down to p from above
    lab[y0, x0 - 1] = 1
    lab[y0, x0 + 1] = 1
    lab[y0 + 1, x0] = 1
    lab[y0 + 1, x0 + 1] = 0         # a 0-cell touching p's ring only at a corner
    lab[y0 + 1:, x0 + 1:] = 0
    lab[y0 + 1, x0 + 1:] = 0
    r = constructed_state(lab, [1], (x0, y0))
    assert r.decide(0, x0, y0) == 1
    assert r.decide(1, x0, y0) == 1


def test_a_move_that_splits_its_superpixel_is_refused():
    lab = np.full((16, 16), 3, np.int32)
    x0, y0 = 6, 6
    lab[:, x0] = 0                  # a vertical line of 0 through p
    lab[y0, x0 - 1] = 1
    lab[y0, x0 + 1] = 1
    r = constructed_state(lab, [1], (x0, y0))
    # moving p to 1 would be favourable but would cut label 0 in two
    assert r.decide(0, x0, y0) == -1
    assert r.decide(1, x0, y0) == -1
    # join the upper and lower halves through the cells right of p: the ring
    # now holds one run of 0, so the same move is allowed
    lab[y0 - 1:y0 + 2, x0 + 1] = 0
    r = constructed_state(lab, [1], (x0, y0))
    assert r.decide(0, x0, y0) == 1
    assert r.decide(1, x0, y0) == 1


# --------------------------------------------------------------------------
# anytime termination (Sec. 5.4, reading R15)
# --------------------------------------------------------------------------

def paper_op_list(L, iters, means_iters=0):
    """The schedule as ops, written out from Sec. 5: the initialisation;
    for each block level L..1 its iterations of four parity phases, then the
    descent; the pixel level's phases; with means iterations (Sec. 6.5) an op
    that starts them and their phases; the output."""
    ops = [("init",)]
    for level in range(L, -1, -1):
        for _ in range(iters):
            for phase in range(4):
                ops.append(("phase", level, phase))
        if level > 0:
            ops.append(("descend",))
    if means_iters:
        ops.append(("means",))
        for _ in range(means_iters):
            for phase in range(4):
                ops.append(("mphase", phase))
    ops.append(("output",))
    return ops


ANYTIME_CASES = [
    # W, H, K, L, B, iters, image seed, means iterations, compactness
    (37, 29, 6, 2, 4, 1, 11, 0, 0),
    (24, 40, 5, 1, 3, 2, 12, 0, 0),
    (30, 22, 4, 0, 5, 2, 13, 0, 0),
    (33, 25, 5, 1, 4, 1, 14, 2, 10),
]


@pytest.mark.parametrize("case", ANYTIME_CASES)
def test_anytime_prefixes_follow_the_op_list(case):
    W, H, K, L, B, iters, seed, mi, m = case
    img = rgb_noise(W, H, seed)
    ops = paper_op_list(L, iters, mi)
    r = ref.Ref(W, H, K, L, B, iters, means_iters=mi, compactness=m)
    assert r.num_ops() == len(ops)
    for n in range(1, len(ops) + 2):
        got = r.run_ops(img, n)
        want = ref.Ref(W, H, K, L, B, iters, means_iters=mi, compactness=m)
        want.init(img)
        for op in ops[1:n]:
            if op[0] == "phase":
                want.run_phase(op[1], op[2])
            elif op[0] == "mphase":
                want.run_means_phase(op[1])
        assert np.array_equal(got, want.labels()), "prefix of %d ops" % n
        # Sec. 5.4: stopping at any point leaves a valid partition
        assert_valid_partition(got, r.K)
        h, s = r.hist()
        h2, s2 = recount(got, r.bins(), r.K, r.nbins)
        assert np.array_equal(h, h2) and np.array_equal(s, s2)


def test_anytime_one_op_is_the_grid_and_all_ops_the_full_run():
    W, H, K = 45, 31, 9
    img = rgb_noise(W, H, 21)
    r = ref.Ref(W, H, K, 2, 4, 2)
    lab = r.run_ops(img, 1)
    sx = [(i * W) // r.gx for i in range(r.gx + 1)]
    sy = [(i * H) // r.gy for i in range(r.gy + 1)]
    for y in range(H):
        for x in range(W):
            cx = max(i for i in range(r.gx) if sx[i] <= x)
            cy = max(i for i in range(r.gy) if sy[i] <= y)
            assert lab[y, x] == cy * r.gx + cx
    full = ref.Ref(W, H, K, 2, 4, 2).run(img)
    assert np.array_equal(r.run_ops(img, r.num_ops()), full)
    assert np.array_equal(r.run_ops(img, r.num_ops() + 5), full)
    with pytest.raises(ref.OracleError):
        r.run_ops(img, 0)


# --------------------------------------------------------------------------
# LAB colour bins (Sec. 6.2, reading R16)
# --------------------------------------------------------------------------

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def real_lab8(rgb):
    """Real-valued 8-bit L*a*b* codes of uint8 triples: the CIE 1976
    formulas over the sRGB decoding curve and the D65 matrix in float64,
    without the oracle's fixed point."""
    c = rgb.astype(np.float64) / 255.0
    lin = np.where(c <= 0.04045, c / 12.92, ((c + 0.055) / 1.055) ** 2.4)
    m = np.array([[0.4124, 0.3576, 0.1805], [0.2126, 0.7152, 0.0722], [0.0193, 0.1192, 0.9505]])
    t = lin @ (m / m.sum(axis=1, keepdims=True)).T
    d = 6.0 / 29.0
    f = np.where(t > d ** 3, np.cbrt(t), t / (3 * d * d) + 4.0 / 29.0)
    L = 116 * f[..., 1] - 16
    a = 500 * (f[..., 0] - f[..., 1])
    b = 200 * (f[..., 1] - f[..., 2])
    code = np.stack([L * 255 / 100, a + 128, b + 128], axis=-1)
    return np.clip(np.floor(code + 0.5), 0, 255)


def lab_ref():
    return ref.Ref(8, 8, 1, 0, 5, 1, color_space=1)


def test_lab_codes_of_the_textbook_colours():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lab_srgb_d65.txt")) if l.strip() and l[0] != "#"]
    rgb = np.array([[int(v) for v in r[:3]] for r in rows], np.uint8)
    lab = np.array([[float(v) for v in r[3:]] for r in rows])
    want = np.stack([lab[:, 0] * 255 / 100, lab[:, 1] + 128, lab[:, 2] + 128], axis=1)
    got = lab_ref().lab8(rgb).astype(np.float64)
    assert np.all(np.abs(got - np.clip(np.floor(want + 0.5), 0, 255)) <= 1), got
    assert got[0].tolist() == [255, 128, 128] and got[1].tolist() == [0, 128, 128]


def test_lab_codes_match_the_real_valued_formulas():
    v = np.arange(0, 256, 3)
    rgb = np.stack(np.meshgrid(v, v, v, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.uint8)
    got = lab_ref().lab8(rgb).astype(np.float64)
    want = real_lab8(rgb)
    diff = np.abs(got - want)
    assert diff.max() <= 1
    assert (diff == 0).mean() > 0.999


def test_lab_greys_are_neutral_and_ordered():
    g = np.repeat(np.arange(256, dtype=np.uint8)[:, None], 3, axis=1)
    got = lab_ref().lab8(g).astype(int)
    assert np.all(got[:, 1] == 128) and np.all(got[:, 2] == 128)
    assert np.all(np.diff(got[:, 0]) >= 0) and got[0, 0] == 0 and got[255, 0] == 255


@pytest.mark.parametrize("B", [1, 4, 5, 8])
def test_lab_bins_are_r1_bins_of_the_lab_codes(B):
    W, H = 41, 23
    img = rgb_noise(W, H, 40 + B)
    r = ref.Ref(W, H, 6, 1, B, 1, color_space=1)
    r.init(img)
    code = r.lab8(img).astype(np.int64)
    q = code * B // 256
    assert np.array_equal(r.bins(), q[..., 0] * B * B + q[..., 1] * B + q[..., 2])
    rgb_bins = ref.Ref(W, H, 6, 1, B, 1)
    rgb_bins.init(img)
    qq = img.astype(np.int64) * B // 256
    assert np.array_equal(rgb_bins.bins(), qq[..., 0] * B * B + qq[..., 1] * B + qq[..., 2])


# --------------------------------------------------------------------------
# means-based pixel updates (SPM, Sec. 6.3 and 6.5; reading R17)
# --------------------------------------------------------------------------

U32 = Fraction(1, 1 << 24)  # unit roundoff of IEEE single precision


def exact_means_decision(labels, codes, K, m, x, y):
    """The means rule in exact fractions: sums recounted from the labels,
    SLIC's distance with (m/S)^2 = m^2 K / N.  Returns (target or -1, the
    exact distances of k and of each candidate, and for each a bound on the
    error of the oracle's single-precision evaluation of it).

    The bound follows the oracle's order of operations (R17): r = 1/n, then
    t = c - S r for each colour and coordinate term, the squares summed, the
    spatial sum scaled by the rounded weight.  Each rounding is at most u =
    2^-24 relative; with mu = S/n the computed t is within about 3u(|mu|+|t|)
    of the exact one, so each squared term is within about 9u(|t|+|mu|)^2
    and the whole distance within 32u times the sum of those squares
    (a generous constant for the adds and the weight's own rounding)."""
    H, W = labels.shape
    k = int(labels[y, x])
    cand = brute.candidates(labels, x, y)
    if not cand or not brute.ring_connected(labels, x, y, k):
        return -1, None, None
    w = Fraction(m * m * K, W * H)

    def dist(lbl):
        ys, xs = np.nonzero(labels == lbl)
        n = len(xs)
        d, scale = Fraction(0), Fraction(0)
        for q in range(3):
            mu = Fraction(int(codes[ys, xs, q].sum()), n)
            t = Fraction(int(codes[y, x, q])) - mu
            d += t * t
            scale += (abs(t) + abs(mu)) ** 2
        for v, tot in ((x, int(xs.sum())), (y, int(ys.sum()))):
            mu = Fraction(tot, n)
            t = v - mu
            d += w * t * t
            scale += (w + 1) * (abs(t) + abs(mu)) ** 2
        return d, 32 * U32 * scale

    dk = dist(k)
    dc = {c: dist(c) for c in cand}
    best = min(cand, key=lambda c: (dc[c][0], c))
    return (best if dc[best][0] < dk[0] else -1), dk, dc


@pytest.mark.parametrize("seed,m,color", [(1, 0, 0), (2, 10, 0), (3, 40, 1), (4, 3, 1)])
def test_means_decisions_match_exact_fractions(seed, m, color):
    """Every decision whose exact distance gaps (k against the best
    candidate, the best against every other candidate) exceed the sum of
    the two distances' rounding bounds equals the exact rule; only those
    within the bounds may go either way, and they are few."""
    W, H, K = 26, 20, 6
    img = rgb_noise(W, H, 60 + seed, 40, 220)
    r = ref.Ref(W, H, K, 1, 4, 1, color_space=color, means_iters=1, compactness=m)
    r.run_ops(img, 1 + 2 * (4 + 1))  # grid, the block level and the histogram pixel phases
    labels = r.labels()
    codes = r.lab8(img) if color else img
    checked = moved = close = 0
    for y in range(H):
        for x in range(W):
            want, dk, dc = exact_means_decision(labels, codes, r.K, m, x, y)
            if dk is None:
                assert r.decide_means(x, y) == -1, (x, y)
                continue
            best = min(dc, key=lambda c: (dc[c][0], c))
            pairs = [(dk, dc[best])] + [(dc[c], dc[best]) for c in dc if c != best]
            if any(abs(a[0] - b[0]) <= a[1] + b[1] for a, b in pairs):
                close += 1
                continue  # within the rounding bounds: either decision is a correct rounding
            assert r.decide_means(x, y) == want, (x, y)
            checked += 1
            moved += want >= 0
    assert moved > 0, "no pixel wanted to move"
    assert close <= max(2, checked // 20), (close, checked)


def two_region_state(m):
    """8 x 4 image, K = 2 (left and right halves); column x = 3 of the left
    superpixel has the right superpixel's colour."""
    img = np.zeros((4, 8, 3), np.uint8)
    img[:, 3:] = 200
    r = ref.Ref(8, 4, 2, 0, 4, 1, patch=0, means_iters=1, compactness=m)
    r.init(img)
    assert r.gx == 2 and r.gy == 1
    return r


def test_means_move_to_the_nearer_colour_mean():
    r = two_region_state(0)
    assert r.decide_means(3, 0) == 1 and r.decide_means(3, 1) == 1
    assert r.decide_means(2, 1) == -1  # already nearest to its own mean
    r.run_means_phase(1)  # phase (py, px) = (0, 1): x odd, y even
    assert r.labels()[0, 3] == 1 and r.labels()[2, 3] == 1


def test_means_compactness_keeps_pixels_near_their_centroid():
    r = two_region_state(1024)  # (m/S)^2 = 1024^2 * 2 / 32: the spatial term dominates
    assert r.decide_means(3, 0) == -1 and r.decide_means(3, 1) == -1


@pytest.mark.parametrize("seed", range(3))
def test_invariants_after_every_means_phase(seed):
    W, H = 31, 23
    img = rgb_noise(W, H, 80 + seed)
    r = ref.Ref(W, H, 7, 1, 3, 1, means_iters=2, compactness=5 * seed)
    r.run_ops(img, r.num_ops() - 1 - 8)  # up to the start of the means iterations
    bins = r.bins()
    moved = 0
    for _ in range(2):
        for phase in range(4):
            moved += r.run_means_phase(phase)
            lab = r.labels()
            h, s = r.hist()
            h2, s2 = recount(lab, bins, r.K, r.nbins)
            assert np.array_equal(h, h2) and np.array_equal(s, s2)
            assert_valid_partition(lab, r.K)
    assert moved > 0


def test_zero_means_iterations_leave_the_run_unchanged():
    W, H = 35, 27
    img = rgb_noise(W, H, 90)
    a = ref.Ref(W, H, 6, 1, 4, 2).run(img)
    b = ref.Ref(W, H, 6, 1, 4, 2, means_iters=0, compactness=30).run(img)
    c = ref.Ref(W, H, 6, 1, 4, 2, means_iters=1).run(img)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_means_equal_candidates_go_to_the_smallest_label():
    # p = (4, 1) is bright in a dark superpixel 0; its neighbours 1 and 2 are
    # both entirely bright, so their means tie exactly
    labels = np.array([[0] * 9, [1, 1, 1, 1, 0, 2, 2, 2, 2], [1, 1, 1, 1, 1, 2, 2, 2, 2]], np.int32)
    img = np.repeat(np.where(labels == 0, 0, 200)[..., None], 3, axis=2).astype(np.uint8)
    img[1, 4] = 200
    r = ref.Ref(9, 3, 3, 0, 4, 1, patch=0, means_iters=1)
    r.init(img)
    assert r.K == 3
    r.set_labels(labels)
    assert r.decide_means(4, 1) == 1


# --------------------------------------------------------------------------
# edge snapping (the edge prior of Sec. 6.4, reading R18)
# --------------------------------------------------------------------------

def frozen_mask(labels, codes, tau):
    """Pixels with a 4-neighbour of another label whose colour codes differ
    by at least tau in L1 (restated with numpy)."""
    c = codes.astype(np.int64)
    H, W = labels.shape
    f = np.zeros((H, W), bool)
    dh = np.abs(c[:, 1:] - c[:, :-1]).sum(axis=2) >= tau
    eh = dh & (labels[:, 1:] != labels[:, :-1])
    f[:, 1:] |= eh
    f[:, :-1] |= eh
    dv = np.abs(c[1:, :] - c[:-1, :]).sum(axis=2) >= tau
    ev = dv & (labels[1:, :] != labels[:-1, :])
    f[1:, :] |= ev
    f[:-1, :] |= ev
    return f


@pytest.mark.parametrize("seed,tau,color", [(1, 250, 0), (2, 300, 0), (3, 120, 1), (4, 200, 1)])
def test_edge_snapped_decisions_are_the_plain_ones_unless_frozen(seed, tau, color):
    W, H, K = 30, 22, 7
    img = rgb_noise(W, H, 200 + seed, 30, 230)
    plain = ref.Ref(W, H, K, 1, 4, 1, color_space=color, means_iters=1, compactness=3)
    plain.run_ops(img, 1 + 2 * 5)  # a state after some block and pixel phases
    labels = plain.labels()
    snap = ref.Ref(W, H, K, 1, 4, 1, color_space=color, means_iters=1, compactness=3, edge_threshold=tau)
    snap.init(img)
    snap.set_labels(labels)
    codes = plain.lab8(img) if color else img
    frozen = frozen_mask(labels, codes, tau)
    n_frozen = n_moving = 0
    for y in range(H):
        for x in range(W):
            want = plain.decide(0, x, y)
            got = snap.decide(0, x, y)
            want_m, got_m = plain.decide_means(x, y), snap.decide_means(x, y)
            if frozen[y, x]:
                assert got == -1 and got_m == -1, (x, y)
                n_frozen += want >= 0
            else:
                assert got == want and got_m == want_m, (x, y)
                n_moving += want >= 0
    assert n_frozen > 0 and n_moving > 0, "the case must hold both kinds"


def test_frozen_pixels_keep_their_labels_through_every_pixel_phase():
    W, H = 36, 28
    img = rgb_noise(W, H, 210, 0, 256)
    tau = 200
    r = ref.Ref(W, H, 8, 2, 4, 2, edge_threshold=tau)
    r.run_ops(img, 1 + 2 * (8 + 1))  # grid and both block levels
    held = 0
    for _ in range(2):
        for phase in range(4):
            before = r.labels()
            frozen = frozen_mask(before, img, tau)
            r.run_phase(0, phase)
            after = r.labels()
            assert np.array_equal(after[frozen], before[frozen])
            held += int(frozen.sum())
    assert held > 0


def test_threshold_above_every_edge_changes_nothing():
    W, H = 33, 25
    img = rgb_noise(W, H, 220, 60, 200)  # no two pixels differ by 3 * 140 = 420 or more
    a = ref.Ref(W, H, 6, 1, 4, 2).run(img)
    b = ref.Ref(W, H, 6, 1, 4, 2, edge_threshold=421).run(img)
    c = ref.Ref(W, H, 6, 1, 4, 2, edge_threshold=30).run(img)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


# --------------------------------------------------------------------------
# compactness prior (Sec. 6.4; reading R19)
# --------------------------------------------------------------------------

def exact_compact_decision(labels, bins, nbins, x, y, gamma, patch, omega):
    """The pixel rule with the compactness prior in exact fractions, in the
    units of the intersection (Prop. 1): every option scores its colour
    term (a one-pixel intersection), gamma times half the exact change of G
    (Eq. 7, Prop. 2) for a candidate, and loses (omega/16) (K/N) d^2, d^2
    the squared distance of the pixel to the option's centre of gravity
    (recounted from the labels; the stay option keeps the pixel).  Returns
    (target or -1, the stay option's (score, bound), each candidate's
    (score, bound)), or (-1, None, None) for a pixel that may not leave.

    The bound covers the oracle's single-precision evaluation (R19: 81 a/s,
    plus gamma G, minus the rounded weight times d^2 from 1/n-scaled sums;
    G <= 90), divided by 81 into these units: 32u (u = 2^-24) times
    81 a/s + 90 gamma + 81 w (|g|+|mu|)^2 summed over both coordinates."""
    H, W = labels.shape
    k = int(labels[y, x])
    cand = brute.candidates(labels, x, y)
    if not cand or not brute.ring_connected(labels, x, y, k):
        return -1, None, None
    K = int(labels.max()) + 1
    w = Fraction(omega, 16) * Fraction(K, W * H)
    j = int(bins[y, x])
    g = Fraction(gamma[0], gamma[1]) if patch else Fraction(0)

    def centre(lbl):
        ys, xs = np.nonzero(labels == lbl)
        n = len(xs)
        d2, sc = Fraction(0), Fraction(0)
        for v, tot in ((x, int(xs.sum())), (y, int(ys.sum()))):
            mu = Fraction(tot, n)
            d2 += (v - mu) ** 2
            sc += (abs(v - mu) + abs(mu)) ** 2
        return d2, sc

    def colour(lbl, without_p):
        sel = labels == lbl
        a, s = int((bins[sel] == j).sum()), int(sel.sum())
        return Fraction(a - 1, s - 1) if without_p else Fraction(a, s)

    def option(col, gterm, lbl):
        d2, sc = centre(lbl)
        bound = 32 * U32 * (81 * col + 90 * g + 81 * w * sc) / 81
        return col + gterm - w * d2, bound

    stay = option(colour(k, True), 0, k)
    scores = {n: option(colour(n, False), g * brute.delta_G(labels, x, y, n) / 2, n) for n in cand}
    best = max(cand, key=lambda n: (scores[n][0], -n))
    return (best if scores[best][0] > stay[0] else -1), stay, scores


@pytest.mark.parametrize("seed,omega,gamma,patch", [(1, 16, (1, 1), 3), (2, 160, (1, 1), 3), (3, 40, (2, 3), 0),
                                                    (4, 1024, (1, 1), 3)])
def test_compact_prior_decisions_match_exact_fractions(seed, omega, gamma, patch):
    """Every decision whose exact score gaps (the best candidate against
    the stay option and against every other candidate) exceed the sum of
    the two scores' rounding bounds equals the exact rule; the few within
    the bounds may go either way."""
    W, H, K = 26, 20, 6
    img = synth.make_image(synth.ImageSpec(W, H, seed=300 + seed, cells=5, sigma=20.0))
    r = ref.Ref(W, H, K, 1, 4, 1, patch, gamma, compact_prior=omega)
    r.run_ops(img, 1 + 4 + 1 + seed % 4)  # the grid, the block level and a few pixel phases
    labels, bins = r.labels(), r.bins()
    checked = moved = close = 0
    for y in range(H):
        for x in range(W):
            want, stay, scores = exact_compact_decision(labels, bins, r.nbins, x, y, gamma, patch, omega)
            if stay is None:
                assert r.decide(0, x, y) == -1, (x, y)
                continue
            best = max(scores, key=lambda n: (scores[n][0], -n))
            pairs = [(stay, scores[best])] + [(scores[n], scores[best]) for n in scores if n != best]
            if any(abs(a[0] - b[0]) <= a[1] + b[1] for a, b in pairs):
                close += 1
                continue  # within the rounding bounds: either decision is a correct rounding
            assert r.decide(0, x, y) == want, (x, y)
            checked += 1
            moved += want >= 0
    assert checked > 20 and moved > 0
    assert close <= max(2, checked // 20), (close, checked)


def strips(x_split, omega, patch=0):
    """12 x 4 constant image, K = 2; the left superpixel is columns
    0..x_split-1 (set by hand), the right one the rest."""
    img = np.full((4, 12, 3), 90, np.uint8)
    r = ref.Ref(12, 4, 2, 0, 4, 1, patch, (1, 1), compact_prior=omega)
    r.init(img)
    assert (r.gx, r.gy) == (2, 1)
    lab = np.zeros((4, 12), np.int32)
    lab[:, x_split:] = 1
    r.set_labels(lab)
    return r


def test_compact_prior_moves_a_pixel_to_the_nearer_centre():
    """One colour everywhere: the colour terms tie, so the prior alone
    decides.  Left superpixel columns 0..8 (centre x = 4), right 9..11
    (centre x = 10): column 8 is nearer the right centre and moves, column 9
    stays, and without the prior nothing moves (strict gain)."""
    r = strips(9, 64)
    for y in range(4):
        assert r.decide(0, 8, y) == 1
        assert r.decide(0, 9, y) == -1
        assert r.decide(0, 7, y) == -1  # not on the boundary
    assert all(strips(9, 0).decide(0, 8, y) == -1 for y in range(4))


def test_compact_prior_pixel_nearer_its_own_centre_stays():
    """Left superpixel columns 0..5 (centre 2.5), right 6..11 (centre 8.5):
    column 5 is 2.5 from its own centre and 3.5 from the right one."""
    r = strips(6, 64)
    assert all(r.decide(0, 5, y) == -1 for y in range(4))
    assert all(r.decide(0, 6, y) == -1 for y in range(4))


def spread(labels):
    """Mean squared distance of the pixels to their superpixel's centre."""
    H, W = labels.shape
    ys, xs = np.mgrid[0:H, 0:W]
    total = 0.0
    for k in np.unique(labels):
        sel = labels == k
        total += ((xs[sel] - xs[sel].mean()) ** 2 + (ys[sel] - ys[sel].mean()) ** 2).sum()
    return total / (W * H)


def test_compact_prior_makes_superpixels_more_compact():
    W, H = 96, 72
    img = synth.make_image(synth.ImageSpec(W, H, seed=77, cells=9, sigma=10.0, texture=True))
    s = [spread(ref.Ref(W, H, 24, 2, 5, 2, compact_prior=w).run(img)) for w in (0, 64, 512)]
    assert s[0] > s[1] > s[2], s


@pytest.mark.parametrize("seed", range(2))
def test_invariants_after_every_phase_with_the_compact_prior(seed):
    W, H = 37, 29
    img = rgb_noise(W, H, 120 + seed)
    r = ref.Ref(W, H, 8, 1, 3, 2, compact_prior=48 * (seed + 1))
    r.init(img)
    bins = r.bins()
    for level, phase in r.schedule():
        r.run_phase(level, phase)
        lab = r.labels()
        h, s = r.hist()
        h2, s2 = recount(lab, bins, r.K, r.nbins)
        assert np.array_equal(h, h2) and np.array_equal(s, s2)
        assert_valid_partition(lab, r.K)


def test_compact_prior_leaves_the_block_levels_alone():
    W, H = 64, 48
    img = synth.make_image(synth.ImageSpec(W, H, seed=78, cells=7, sigma=12.0))
    nblock = 1 + 2 * (4 * 2 + 1)  # the grid and two block levels of two iterations, with their descents
    a = ref.Ref(W, H, 12, 2, 4, 2)
    b = ref.Ref(W, H, 12, 2, 4, 2, compact_prior=512)
    assert np.array_equal(a.run_ops(img, nblock), b.run_ops(img, nblock))
    assert not np.array_equal(a.run(img), b.run(img))


# --------------------------------------------------------------------------
# SPM on its own (Sec. 6.3; reading R20)
# --------------------------------------------------------------------------

def test_spm_alone_starts_the_means_iterations_from_the_grid():
    W, H = 40, 30
    img = synth.make_image(synth.ImageSpec(W, H, seed=79, cells=6, sigma=10.0))
    r = ref.Ref(W, H, 10, 2, 4, 0, means_iters=2, compactness=8)
    grid = ref.Ref(W, H, 10, 2, 4, 1)
    grid.init(img)
    # init and the two descents leave the grid as it is
    assert np.array_equal(r.run_ops(img, 1 + 2), grid.labels())
    assert r.num_ops() == 1 + 2 + 1 + 4 * 2 + 1
    # the means phases from the grid, against their exact-fraction rule
    r.run_ops(img, 1 + 2 + 1)
    labels, codes = r.labels(), img
    moved = 0
    for y in range(H):
        for x in range(W):
            want, dk, dc = exact_means_decision(labels, codes, r.K, 8, x, y)
            if dk is not None:
                best = min(dc, key=lambda c: (dc[c][0], c))
                pairs = [(dk, dc[best])] + [(dc[c], dc[best]) for c in dc if c != best]
                if any(abs(a[0] - b[0]) <= a[1] + b[1] for a, b in pairs):
                    continue  # within the single-precision rounding bounds
            assert r.decide_means(x, y) == want, (x, y)
            moved += want >= 0
    assert moved > 0
    full = r.run(img)
    assert not np.array_equal(full, grid.labels())
    # the whole run is the means phases applied to the grid, nothing else
    m = ref.Ref(W, H, 10, 2, 4, 0, means_iters=2, compactness=8)
    m.init(img)
    for _ in range(2):
        for phase in range(4):
            m.run_means_phase(phase)
    assert np.array_equal(full, m.labels())


def test_no_iterations_at_all_is_refused():
    assert ref.grid(40, 30, 10, 2, 4, 0)[0] == ref.EINVAL
