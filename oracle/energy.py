"""The SEEDS energy E(s) = H(s) + gamma*G(s) written out from its definitions,
in exact fractions.  TEST INFRASTRUCTURE (small images only).

  c_{A_k}(j) = (1/|A_k|) * #{i in A_k : I(i) in bin j}     Eq. 4 (Z = |A_k|)
  H(s)       = sum_k sum_j c_{A_k}(j)^2                    Eqs. 3 and 5
  b_{N_i}(k) = (1/Z) * #{q in N_i : s(q) = k}, Z = 9       Eq. 6
  G(s)       = sum_i sum_k b_{N_i}(k)^2                    Eq. 7
  E(s)       = H(s) + gamma * G(s)                         Eq. 2

N_i is the 3x3 patch around pixel i clipped to the image; Z stays 9 at the
border (the normalisation the paper's Prop. 2 needs to be exact).
"""
from fractions import Fraction

import numpy as np

Z_PATCH = 9


def colour_term(labels: np.ndarray, bins: np.ndarray) -> Fraction:
    """H(s) for a label map and the per-pixel colour bins."""
    counts = {}
    sizes = {}
    for k, j in zip(labels.ravel().tolist(), bins.ravel().tolist()):
        counts[(k, j)] = counts.get((k, j), 0) + 1
        sizes[k] = sizes.get(k, 0) + 1
    H = Fraction(0)
    for (k, j), c in counts.items():
        H += Fraction(c, sizes[k]) ** 2
    return H


def patch_histogram(labels: np.ndarray, x: int, y: int) -> dict:
    """b_{N_i} for i = (x, y), in counts (multiply by 1/Z for Eq. 6)."""
    Hh, Ww = labels.shape
    b = {}
    for qy in range(y - 1, y + 2):
        for qx in range(x - 1, x + 2):
            if 0 <= qx < Ww and 0 <= qy < Hh:
                k = int(labels[qy, qx])
                b[k] = b.get(k, 0) + 1
    return b


def boundary_term_counts(labels: np.ndarray) -> int:
    """Z^2 * G(s) = sum_i sum_k (#{q in N_i : s(q)=k})^2, an integer."""
    Hh, Ww = labels.shape
    total = 0
    for y in range(Hh):
        for x in range(Ww):
            total += sum(c * c for c in patch_histogram(labels, x, y).values())
    return total


def boundary_term(labels: np.ndarray) -> Fraction:
    """G(s) of Eq. 7."""
    return Fraction(boundary_term_counts(labels), Z_PATCH * Z_PATCH)


def energy(labels: np.ndarray, bins: np.ndarray, gamma: Fraction, patch: int = 3) -> Fraction:
    """E(s) of Eq. 2; patch == 0 drops the boundary term."""
    E = colour_term(labels, bins)
    if patch:
        E += Fraction(gamma) * boundary_term(labels)
    return E
