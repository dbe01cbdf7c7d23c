"""Brute-force restatement of one phase's decisions, for pinning the oracle.

Independent of the oracle's C code: histograms are recounted from the labels,
the colour test is the paper's intersection distance on NORMALISED
histograms (Sec. 5.3, Prop. 1) in exact fractions, the boundary term's change
is recounted from the definition of G (Eq. 7) rather than taken from Prop. 2,
and connectivity is a breadth-first search over the ring instead of the
oracle's run walk.  Tiny images only.

Scores (the reading of how the two proxies add up): a block compares
int(c_An, c_L) against int(c_{Ak\\L}, c_L); a pixel adds gamma/2 times the
exact change of G to the intersection term.  Prop. 2 makes the latter equal
to the counted form gamma*(G_n + |K_p| - G_k)/81 used by the oracle, since
Z^2 * dG = 2*(G_n + |K_p| - G_k) with Z = 9.
"""
from fractions import Fraction

import numpy as np

from oracle import energy


def normalised_hist(bins_of_set, nbins):
    n = len(bins_of_set)
    h = [0] * nbins
    for j in bins_of_set:
        h[j] += 1
    return [Fraction(c, n) for c in h]


def intersection(a, b):
    return sum((min(x, y) for x, y in zip(a, b)), Fraction(0))


def unit_grid_labels(labels, xe, ye):
    return labels[np.ix_(ye[:-1], xe[:-1])]


def ring_connected(grid, bx, by, k):
    """Rule: some 4-neighbour is k, and every k 4-neighbour is reachable from
    every other through k-labelled cells of the 8-ring (4-adjacency)."""
    nby, nbx = grid.shape
    ring = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]

    def is_k(dx, dy):
        x, y = bx + dx, by + dy
        return 0 <= x < nbx and 0 <= y < nby and grid[y, x] == k

    kcells = {c for c in ring if is_k(*c)}
    four = [c for c in [(-1, 0), (1, 0), (0, -1), (0, 1)] if c in kcells]
    if not four:
        return False
    seen = {four[0]}
    todo = [four[0]]
    while todo:
        cx, cy = todo.pop()
        for nx, ny in ((cx - 1, cy), (cx + 1, cy), (cx, cy - 1), (cx, cy + 1)):
            if (nx, ny) in kcells and (nx, ny) not in seen:
                seen.add((nx, ny))
                todo.append((nx, ny))
    return all(c in seen for c in four)


def candidates(grid, bx, by):
    nby, nbx = grid.shape
    k = grid[by, bx]
    out = set()
    for x, y in ((bx - 1, by), (bx + 1, by), (bx, by - 1), (bx, by + 1)):
        if 0 <= x < nbx and 0 <= y < nby and grid[y, x] != k:
            out.add(int(grid[y, x]))
    return sorted(out)


def local_patch_sumsq(labels, x0, x1, y0, y1):
    Hh, Ww = labels.shape
    t = 0
    for y in range(max(0, y0 - 1), min(Hh, y1 + 1)):
        for x in range(max(0, x0 - 1), min(Ww, x1 + 1)):
            t += sum(c * c for c in energy.patch_histogram(labels, x, y).values())
    return t


def delta_G(labels, x, y, n):
    """Exact change of G (Eq. 7) if pixel (x,y) takes label n."""
    before = local_patch_sumsq(labels, x, x + 1, y, y + 1)
    old = labels[y, x]
    labels[y, x] = n
    after = local_patch_sumsq(labels, x, x + 1, y, y + 1)
    labels[y, x] = old
    return Fraction(after - before, 81)


def phase_decisions(labels, bins, nbins, level, phase, xe, ye, gamma, patch):
    """{(bx,by): n} for every unit of the phase that moves."""
    labels = labels.copy()
    grid = unit_grid_labels(labels, xe, ye)
    nby, nbx = grid.shape
    K = int(labels.max()) + 1
    members = {}
    for k, j in zip(labels.ravel().tolist(), bins.ravel().tolist()):
        members.setdefault(k, []).append(j)
    py, px = phase >> 1, phase & 1
    out = {}
    gamma = Fraction(gamma[0], gamma[1])
    for by in range(py, nby, 2):
        for bx in range(px, nbx, 2):
            k = int(grid[by, bx])
            cands = candidates(grid, bx, by)
            if not cands or not ring_connected(grid, bx, by, k):
                continue
            x0, x1, y0, y1 = xe[bx], xe[bx + 1], ye[by], ye[by + 1]
            Lbins = bins[y0:y1, x0:x1].ravel().tolist()
            cL = normalised_hist(Lbins, nbins)
            rest = list(members[k])
            for j in Lbins:
                rest.remove(j)
            stay = intersection(normalised_hist(rest, nbins), cL)
            scores = {}
            for n in cands:
                s = intersection(normalised_hist(members[n], nbins), cL)
                if level == 0 and patch:
                    s += gamma * delta_G(labels, bx, by, n) / 2
                scores[n] = s
            best = max(scores.values())
            n_best = min(n for n in cands if scores[n] == best)
            if scores[n_best] > stay:
                out[(bx, by)] = n_best
    assert K >= 1
    return out


def apply_decisions(labels, decisions, xe, ye):
    out = labels.copy()
    for (bx, by), n in decisions.items():
        out[ye[by]:ye[by + 1], xe[bx]:xe[bx + 1]] = n
    return out
