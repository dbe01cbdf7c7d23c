"""Superpixel quality metrics of Sec. 6.1 against a ground-truth
segmentation (host numpy): undersegmentation error (UE, Sec. 6.1.1),
corrected undersegmentation error (CUE, Sec. 6.1.2), boundary recall (BR,
tolerance epsilon = 2 pixels, Sec. 6.1.3) and achievable segmentation
accuracy (ASA, Sec. 6.1.4).  Labels and truth are integer H x W arrays."""
import numpy as np
from scipy import ndimage


def _overlap(labels, truth):
    """Counts n[k, i] = |s_k intersect g_i|."""
    K, G = int(labels.max()) + 1, int(truth.max()) + 1
    n = np.zeros((K, G), np.int64)
    np.add.at(n, (labels.ravel(), truth.ravel()), 1)
    return n


def ue(labels, truth):
    n = _overlap(labels, truth)
    size = n.sum(axis=1)
    # sum over g_i and over s_k meeting g_i of |s_k - g_i|
    err = sum(int((size[n[:, i] > 0] - n[n[:, i] > 0, i]).sum()) for i in range(n.shape[1]))
    return err / labels.size


def cue(labels, truth):
    n = _overlap(labels, truth)
    return float((n.sum(axis=1) - n.max(axis=1)).sum()) / labels.size


def asa(labels, truth):
    return float(_overlap(labels, truth).max(axis=1).sum()) / labels.size


def boundary(labels):
    """Pixels with a 4-neighbour of another label."""
    b = np.zeros(labels.shape, bool)
    d = labels[:, 1:] != labels[:, :-1]
    b[:, 1:] |= d
    b[:, :-1] |= d
    d = labels[1:, :] != labels[:-1, :]
    b[1:, :] |= d
    b[:-1, :] |= d
    return b


def br(labels, truth, eps=2.0):
    bg, bs = boundary(truth), boundary(labels)
    if not bg.any():
        return 1.0
    dist = ndimage.distance_transform_edt(~bs)  # distance to the nearest superpixel boundary pixel
    return float((dist[bg] < eps).mean())
