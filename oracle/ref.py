"""ctypes access to the C oracle (seeds_ref.c).  TEST INFRASTRUCTURE.

Every call runs the plain CPU code of seeds_ref.c; nothing here computes
anything of the method itself.  Arrays go in and out as numpy arrays.
"""
import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

OK, EINVAL, EGEOM, ENOMEM, ESIZE = 0, -1, -2, -4, -7


class RefParams(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("num_superpixels", ctypes.c_int32),
        ("block_levels", ctypes.c_int32),
        ("bins_per_channel", ctypes.c_int32),
        ("iters_per_level", ctypes.c_int32),
        ("patch", ctypes.c_int32),
        ("gamma_num", ctypes.c_int32),
        ("gamma_den", ctypes.c_int32),
        ("color_space", ctypes.c_int32),
        ("means_iters", ctypes.c_int32),
        ("compactness", ctypes.c_int32),
        ("edge_threshold", ctypes.c_int32),
        ("compact_prior", ctypes.c_int32),
    ]


def lib():
    """Load (building first if needed) the oracle library."""
    global _lib
    with _lock:
        if _lib is None:
            # SEEDS_REF_LIB points the tests at a deliberately broken build
            # of the oracle (mutation tests of the pins); unset otherwise
            path = os.environ.get("SEEDS_REF_LIB") or _build.build()
            L = ctypes.CDLL(path)
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            P = ctypes.POINTER
            L.ref_check_params.argtypes = [P(RefParams)]
            L.ref_grid.argtypes = [P(RefParams), P(i32), P(i32)]
            L.ref_create.argtypes = [P(RefParams), P(vp)]
            L.ref_destroy.argtypes = [vp]
            L.ref_destroy.restype = None
            L.ref_info.argtypes = [vp, P(i32), P(i32), P(i32), P(i32)]
            L.ref_level_grid.argtypes = [vp, ctypes.c_int, P(i32), P(i32), vp, vp]
            L.ref_init.argtypes = [vp, vp, i64]
            L.ref_run_phase.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.ref_run_phase.restype = i64
            L.ref_run.argtypes = [vp, vp, i64]
            L.ref_run.restype = i64
            L.ref_run_ops.argtypes = [vp, vp, i64, i32]
            L.ref_run_ops.restype = i64
            L.ref_num_ops.argtypes = [vp]
            L.ref_num_ops.restype = i32
            L.ref_run_means_phase.argtypes = [vp, ctypes.c_int]
            L.ref_run_means_phase.restype = i64
            L.ref_decide_means.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.ref_lab8.argtypes = [vp, vp, i64, vp]
            L.ref_lab8.restype = None
            L.ref_get_labels.argtypes = [vp, vp]
            L.ref_get_labels.restype = None
            L.ref_get_bins.argtypes = [vp, vp]
            L.ref_get_bins.restype = None
            L.ref_get_hist.argtypes = [vp, vp, vp]
            L.ref_get_hist.restype = None
            L.ref_set_labels.argtypes = [vp, vp]
            L.ref_patch_label_count.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(i64)]
            L.ref_patch_label_count.restype = i64
            L.ref_decide.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.ref_run_sequential.argtypes = [vp, vp, i64, u64, ctypes.c_int, vp, i64]
            L.ref_run_sequential.restype = i64
            L.ref_splitmix64_draws.argtypes = [u64, i32, vp]
            L.ref_splitmix64_draws.restype = None
            L.ref_unit_order.argtypes = [u64, i32, vp]
            L.ref_unit_order.restype = None
            L.ref_candidate_picks.argtypes = [u64, i32, i32, vp]
            L.ref_candidate_picks.restype = None
            _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with status %d" % (what, code))
        self.code = code


def make_params(width, height, num_superpixels, block_levels, bins_per_channel, iters_per_level,
                patch=3, gamma=(1, 1), color_space=0, means_iters=0, compactness=0, edge_threshold=0,
                compact_prior=0):
    return RefParams(int(width), int(height), int(num_superpixels), int(block_levels), int(bins_per_channel),
                     int(iters_per_level), int(patch), int(gamma[0]), int(gamma[1]), int(color_space),
                     int(means_iters), int(compactness), int(edge_threshold), int(compact_prior))


def grid(width, height, num_superpixels, block_levels=0, bins_per_channel=5, iters_per_level=1, patch=3,
         gamma=(1, 1)):
    """(status, gx, gy) for a parameter set."""
    p = make_params(width, height, num_superpixels, block_levels, bins_per_channel, iters_per_level, patch, gamma)
    gx, gy = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib().ref_grid(ctypes.byref(p), ctypes.byref(gx), ctypes.byref(gy))
    return rc, gx.value, gy.value


def splitmix64_draws(seed, n):
    """The first n 64-bit draws of the sequential mode's generator from
    state `seed`."""
    out = np.zeros(n, np.uint64)
    lib().ref_splitmix64_draws(ctypes.c_uint64(seed), n, out.ctypes.data)
    return [int(v) for v in out]


def unit_order(seed, nu):
    """The sequential mode's first-sweep visiting order of nu units."""
    out = np.zeros(nu, np.int32)
    lib().ref_unit_order(ctypes.c_uint64(seed), nu, out.ctypes.data)
    return out


def candidate_picks(seed, nc, n):
    """n successive candidate picks among nc, as the sequential mode draws
    them from state `seed`."""
    out = np.zeros(n, np.int32)
    lib().ref_candidate_picks(ctypes.c_uint64(seed), nc, n, out.ctypes.data)
    return out


def _rgb_arg(rgb):
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    assert rgb.ndim == 3 and rgb.shape[2] == 3
    return rgb, rgb.shape[1] * 3


class Ref:
    """One image's oracle state."""

    def __init__(self, width, height, num_superpixels, block_levels, bins_per_channel, iters_per_level,
                 patch=3, gamma=(1, 1), color_space=0, means_iters=0, compactness=0, edge_threshold=0,
                 compact_prior=0):
        self.params = make_params(width, height, num_superpixels, block_levels, bins_per_channel,
                                  iters_per_level, patch, gamma, color_space, means_iters, compactness,
                                  edge_threshold, compact_prior)
        self.means_iters = int(means_iters)
        self._h = ctypes.c_void_p()
        rc = lib().ref_create(ctypes.byref(self.params), ctypes.byref(self._h))
        if rc:
            raise OracleError(rc, "ref_create")
        gx, gy, K, nb = (ctypes.c_int32() for _ in range(4))
        lib().ref_info(self._h, ctypes.byref(gx), ctypes.byref(gy), ctypes.byref(K), ctypes.byref(nb))
        self.W, self.H = int(width), int(height)
        self.L, self.iters = int(block_levels), int(iters_per_level)
        self.gx, self.gy, self.K, self.nbins = gx.value, gy.value, K.value, nb.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.ref_destroy(h)
            self._h = None

    # --- geometry -------------------------------------------------------
    def level_grid(self, level):
        """(nbx, nby, x_edges, y_edges) of a level (0 = pixels)."""
        nbx, nby = ctypes.c_int32(), ctypes.c_int32()
        rc = lib().ref_level_grid(self._h, level, ctypes.byref(nbx), ctypes.byref(nby), None, None)
        if rc:
            raise OracleError(rc, "ref_level_grid")
        xe = np.zeros(nbx.value + 1, np.int32)
        ye = np.zeros(nby.value + 1, np.int32)
        lib().ref_level_grid(self._h, level, ctypes.byref(nbx), ctypes.byref(nby),
                             xe.ctypes.data, ye.ctypes.data)
        return nbx.value, nby.value, xe, ye

    def schedule(self):
        """The (level, phase) sequence of the parity schedule."""
        return [(l, ph) for l in range(self.L, -1, -1) for _ in range(self.iters) for ph in range(4)]

    # --- running ----------------------------------------------------------
    def init(self, rgb):
        rgb, stride = _rgb_arg(rgb)
        rc = lib().ref_init(self._h, rgb.ctypes.data, stride)
        if rc:
            raise OracleError(rc, "ref_init")

    def run_means_phase(self, phase):
        n = lib().ref_run_means_phase(self._h, phase)
        if n < 0:
            raise OracleError(n, "ref_run_means_phase")
        return n

    def decide_means(self, x, y):
        """Means-based decision (R17) for pixel (x, y) against the current labels."""
        return lib().ref_decide_means(self._h, x, y)

    def run_phase(self, level, phase):
        n = lib().ref_run_phase(self._h, level, phase)
        if n < 0:
            raise OracleError(n, "ref_run_phase")
        return n

    def run(self, rgb):
        """Whole schedule from the image; returns the pixel labels."""
        rgb, stride = _rgb_arg(rgb)
        n = lib().ref_run(self._h, rgb.ctypes.data, stride)
        if n < 0:
            raise OracleError(n, "ref_run")
        self.total_moves = n
        return self.labels()

    def num_ops(self):
        """Ops of the schedule: init, per block level 4*iters phases and a
        descent, 4*iters pixel phases, the output (Sec. 5.4 reading R15)."""
        return int(lib().ref_num_ops(self._h))

    def run_ops(self, rgb, nops):
        """Anytime termination: the partition after the first nops ops."""
        rgb, stride = _rgb_arg(rgb)
        n = lib().ref_run_ops(self._h, rgb.ctypes.data, stride, int(nops))
        if n < 0:
            raise OracleError(n, "ref_run_ops")
        self.total_moves = n
        return self.labels()

    def sequential(self, rgb, seed, exact=False, trace_cap=1 << 20):
        """Sequential mode; returns (labels, trace[(level, unit, k, n)], n_accepted)."""
        rgb, stride = _rgb_arg(rgb)
        trace = np.zeros((trace_cap, 4), np.int32)
        n = lib().ref_run_sequential(self._h, rgb.ctypes.data, stride, ctypes.c_uint64(seed),
                                     1 if exact else 0, trace.ctypes.data, trace_cap)
        if n < 0:
            raise OracleError(n, "ref_run_sequential")
        return self.labels(), trace[:min(n, trace_cap)].copy(), n

    def decide(self, level, bx, by):
        return lib().ref_decide(self._h, level, bx, by)

    def patch_label_count(self, x, y, label):
        """(sum_{i in K_p} b_{N_i}(label) in counts, |K_p|)."""
        kp = ctypes.c_int64()
        g = lib().ref_patch_label_count(self._h, x, y, label, ctypes.byref(kp))
        return g, kp.value

    # --- state --------------------------------------------------------------
    def labels(self):
        out = np.zeros((self.H, self.W), np.int32)
        lib().ref_get_labels(self._h, out.ctypes.data)
        return out

    def lab8(self, rgb):
        """The 8-bit CIE L*a*b* codes (reading R16) of an (..., 3) uint8 array."""
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        assert rgb.shape[-1] == 3
        out = np.zeros(rgb.shape, np.uint8)
        lib().ref_lab8(self._h, rgb.ctypes.data, rgb.size // 3, out.ctypes.data)
        return out

    def bins(self):
        out = np.zeros((self.H, self.W), np.int32)
        lib().ref_get_bins(self._h, out.ctypes.data)
        return out

    def hist(self):
        h = np.zeros((self.K, self.nbins), np.int64)
        s = np.zeros(self.K, np.int64)
        lib().ref_get_hist(self._h, h.ctypes.data, s.ctypes.data)
        return h, s

    def set_labels(self, labels):
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        assert labels.shape == (self.H, self.W)
        rc = lib().ref_set_labels(self._h, labels.ctypes.data)
        if rc:
            raise OracleError(rc, "ref_set_labels")

    def level_labels(self, level):
        """Label of every unit of a level, read at the unit's first pixel."""
        nbx, nby, xe, ye = self.level_grid(level)
        lab = self.labels()
        return lab[np.ix_(ye[:-1], xe[:-1])]
