"""Thin ctypes binding of libseeds.so (include/seeds.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions carry the C names; `SeedsContext` adds the torch
plumbing (device memory via data_ptr(), streams via cuda_stream).  If the
compiled library is missing this module raises on import -- there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
# SEEDS_LIB selects another build of the library (the bounds-checked debug
# build in its tests); unset, the in-tree libseeds.so
LIB_PATH = os.environ.get("SEEDS_LIB") or os.path.join(_HERE, "libseeds.so")

SEEDS_OK = 0
SEEDS_ERR_INVALID = -1
SEEDS_ERR_GEOMETRY = -2
SEEDS_ERR_INT64 = -3
SEEDS_ERR_NO_MEMORY = -4
SEEDS_ERR_CUDA = -5
SEEDS_ERR_DEVICE = -6
SEEDS_ERR_STATIC_SIZE = -7
SEEDS_STATIC_SCRATCH_BYTES = 32 << 20
SEEDS_MAX_LEVELS = 12
SEEDS_MAX_BATCH = 4096

_NAMES = {0: "SEEDS_OK", -1: "SEEDS_ERR_INVALID", -2: "SEEDS_ERR_GEOMETRY", -3: "SEEDS_ERR_INT64",
          -4: "SEEDS_ERR_NO_MEMORY", -5: "SEEDS_ERR_CUDA", -6: "SEEDS_ERR_DEVICE", -7: "SEEDS_ERR_STATIC_SIZE"}

# every entry point of include/seeds.h
EXPORTS = [
    "seeds_params_default", "seeds_feasible_levels", "seeds_check_params", "seeds_footprint", "seeds_plan",
    "seeds_create",
    "seeds_iterate", "seeds_labels", "seeds_num_superpixels", "seeds_status", "seeds_destroy",
    "seeds_batch_create", "seeds_batch_size", "seeds_batch_num_superpixels", "seeds_batch_iterate",
    "seeds_batch_labels", "seeds_batch_run", "seeds_batch_run_anytime", "seeds_anytime_steps", "seeds_run_host", "seeds_run_host_stream", "seeds_set_tuning", "seeds_get_tuning",
    "seeds_tune_search",
    "seeds_debug_num_ops", "seeds_debug_op_info", "seeds_debug_run_ops", "seeds_debug_read_state",
    "seeds_debug_set_labels", "seeds_debug_inject_error", "seeds_debug_barrier_test", "seeds_debug_launch_count", "seeds_profile_enable",
    "seeds_profile_last_ms", "seeds_profile_steps", "seeds_run_static", "seeds_autotune",
    "seeds_server_create", "seeds_server_destroy", "seeds_server_submit", "seeds_server_step", "seeds_server_poll",
    "seeds_server_drain", "seeds_server_stats",
]


class SeedsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s returned %s (%d)" % (what, _NAMES.get(code, "?"), code))
        self.code = code


class seeds_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("num_superpixels", ctypes.c_int32),
                ("block_levels", ctypes.c_int32), ("bins_per_channel", ctypes.c_int32),
                ("iters_per_level", ctypes.c_int32), ("patch", ctypes.c_int32), ("gamma_num", ctypes.c_int32),
                ("gamma_den", ctypes.c_int32), ("color_space", ctypes.c_int32), ("means_iters", ctypes.c_int32),
                ("compactness", ctypes.c_int32), ("edge_threshold", ctypes.c_int32),
                ("compact_prior", ctypes.c_int32)]


class seeds_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("epoch_steps", ctypes.c_int32),
                ("max_bins_per_channel", ctypes.c_int32)]


class seeds_server_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("resident", ctypes.c_int32), ("arena_free_bytes", ctypes.c_int64),
                ("epochs", ctypes.c_int64), ("launches", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("host_ms", ctypes.c_double)]


class seeds_plan_entry(ctypes.Structure):
    _fields_ = [("img", ctypes.c_int32), ("op", ctypes.c_int32), ("level", ctypes.c_int32),
                ("phase", ctypes.c_int32), ("opidx", ctypes.c_int32), ("units", ctypes.c_int32),
                ("group", ctypes.c_int32), ("cphase", ctypes.c_int32), ("vt_begin", ctypes.c_int64)]


class seeds_tuning(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("hist_layout", ctypes.c_int32), ("small_block_area", ctypes.c_int32),
                ("pixel_tile_rows", ctypes.c_int32), ("block_tiles", ctypes.c_int32)]


TUNE_COST_FN = ctypes.CFUNCTYPE(ctypes.c_float, ctypes.POINTER(seeds_tuning), ctypes.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libseeds.so is not built (expected at %s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "seeds_params_default": [P(seeds_params), i32, i32, i32],
        "seeds_feasible_levels": [P(seeds_params), P(i32)],
        "seeds_check_params": [P(seeds_params), P(i32), P(i32)],
        "seeds_footprint": [P(seeds_params), i32, P(i64)],
        "seeds_plan": [P(seeds_params), i32, P(seeds_tuning), i32, P(i32), P(i32), P(seeds_plan_entry), i32, P(i32),
                       P(i32), P(i64), i32, P(i32)],
        "seeds_create": [P(seeds_params), P(vp)],
        "seeds_iterate": [vp, vp, i64, vp],
        "seeds_labels": [vp, vp, vp],
        "seeds_num_superpixels": [vp, P(i32)],
        "seeds_status": [vp],
        "seeds_destroy": [vp],
        "seeds_batch_create": [P(seeds_params), i32, P(vp)],
        "seeds_batch_size": [vp, P(i32)],
        "seeds_batch_num_superpixels": [vp, i32, P(i32)],
        "seeds_batch_iterate": [vp, P(vp), P(i64), vp],
        "seeds_batch_labels": [vp, P(vp), vp],
        "seeds_batch_run": [vp, P(vp), P(i64), P(vp), vp],
        "seeds_batch_run_anytime": [vp, P(vp), P(i64), P(vp), i32, i64, vp],
        "seeds_anytime_steps": [vp, P(i32)],
        "seeds_run_host": [vp, P(vp), P(i64), P(vp), vp],
        "seeds_run_host_stream": [vp, i32, P(vp), P(i64), P(vp), vp],
        "seeds_set_tuning": [vp, P(seeds_tuning)],
        "seeds_get_tuning": [vp, P(seeds_tuning)],
        "seeds_tune_search": [P(seeds_tuning), TUNE_COST_FN, vp, P(seeds_tuning)],
        "seeds_debug_num_ops": [vp, i32, P(i32)],
        "seeds_debug_op_info": [vp, i32, i32, P(i32), P(i32), P(i32)],
        "seeds_debug_run_ops": [vp, P(vp), P(i64), i32, i32, vp],
        "seeds_debug_read_state": [vp, i32, i32, vp, vp, vp, vp],
        "seeds_debug_set_labels": [vp, i32, i32, vp],
        "seeds_debug_inject_error": [vp],
        "seeds_debug_barrier_test": [vp, i64, i32],
        "seeds_debug_launch_count": [vp, P(i64)],
        "seeds_profile_enable": [vp, i32],
        "seeds_profile_last_ms": [vp, P(ctypes.c_float)],
        "seeds_profile_steps": [vp, vp, i32, P(i32)],
        "seeds_run_static": [P(seeds_params), vp, i64, vp, vp, vp],
        "seeds_autotune": [vp, P(vp), P(i64), P(vp), i32, vp, P(seeds_tuning)],
        "seeds_server_create": [P(seeds_server_config), P(vp)],
        "seeds_server_destroy": [vp],
        "seeds_server_submit": [vp, P(seeds_params), vp, i64, vp, P(i64)],
        "seeds_server_step": [vp, P(i32)],
        "seeds_server_poll": [vp, P(i64), P(ctypes.c_float), i32, P(i32)],
        "seeds_server_drain": [vp],
        "seeds_server_stats": [vp, P(seeds_server_stats_t)],
    }
    for name in EXPORTS:
        f = getattr(L, name)
        f.argtypes = sig[name]
        f.restype = ctypes.c_int
    return L


lib = _load()


def check(code: int, what: str) -> int:
    if code != SEEDS_OK:
        raise SeedsError(code, what)
    return code


def make_params(width, height, num_superpixels, block_levels, bins_per_channel, iters_per_level, patch=3,
                gamma=(1, 1), color_space=0, means_iters=0, compactness=0, edge_threshold=0,
                compact_prior=0) -> seeds_params:
    """color_space: 0 = RGB bytes, 1 = 8-bit CIE L*a*b* codes (Sec. 6.2);
    means_iters / compactness: means-based pixel iterations with SLIC's m
    (Sec. 6.3, 6.5); edge_threshold: edge snapping (Sec. 6.4), 0 = off;
    compact_prior: the compactness prior of Sec. 6.4 in the histogram pixel
    phases, weight compact_prior/16, 0 = off."""
    return seeds_params(int(width), int(height), int(num_superpixels), int(block_levels), int(bins_per_channel),
                        int(iters_per_level), int(patch), int(gamma[0]), int(gamma[1]), int(color_space),
                        int(means_iters), int(compactness), int(edge_threshold), int(compact_prior))


def feasible_levels(width, height, num_superpixels) -> int:
    p = make_params(width, height, num_superpixels, 0, 5, 1)
    out = ctypes.c_int32()
    check(lib.seeds_feasible_levels(ctypes.byref(p), ctypes.byref(out)), "seeds_feasible_levels")
    return out.value


def tune_search(start: seeds_tuning, cost) -> seeds_tuning:
    """The autotuner's search (seeds_tune_search) with a Python cost: cost
    takes a seeds_tuning and returns milliseconds."""
    fn = TUNE_COST_FN(lambda t, _user: float(cost(t.contents)))
    best = seeds_tuning()
    check(lib.seeds_tune_search(ctypes.byref(start), fn, None, ctypes.byref(best)), "seeds_tune_search")
    return best


OP_KINDS = {0: "init", 1: "phase", 2: "descend", 3: "output", 4: "catchup", 5: "means_init", 6: "means_phase"}


def plan(params: Sequence[seeds_params], sm_count: int, tuning: seeds_tuning = None, op_begin=None, op_end=None):
    """The step schedule a launch over these images uses on a GPU with
    sm_count SMs, planned on the host (seeds_plan): a list of steps, each a
    (thread count, [entry dicts]) pair.  op_begin / op_end: per image, the
    ops the launch runs (None = a full run)."""
    n = len(params)
    arr = (seeds_params * n)(*params)
    tp = ctypes.byref(tuning) if tuning is not None else None
    ob = (ctypes.c_int32 * n)(*op_begin) if op_begin is not None else None
    oe = (ctypes.c_int32 * n)(*op_end) if op_end is not None else None
    ne, ns = ctypes.c_int32(), ctypes.c_int32()
    check(lib.seeds_plan(arr, n, tp, sm_count, ob, oe, None, 0, ctypes.byref(ne), None, None, 0, ctypes.byref(ns)),
          "seeds_plan")
    out = (seeds_plan_entry * max(1, ne.value))()
    first = (ctypes.c_int32 * (ns.value + 1))()
    threads = (ctypes.c_int64 * max(1, ns.value))()
    check(lib.seeds_plan(arr, n, tp, sm_count, ob, oe, out, ne.value, ctypes.byref(ne), first, threads,
                         ns.value + 1, ctypes.byref(ns)), "seeds_plan")
    steps = []
    for s in range(ns.value):
        ents = [{f: getattr(out[q], f) for f, _ in seeds_plan_entry._fields_} for q in range(first[s], first[s + 1])]
        steps.append((threads[s], ents))
    return steps


def check_params(p: seeds_params):
    gx, gy = ctypes.c_int32(), ctypes.c_int32()
    rc = lib.seeds_check_params(ctypes.byref(p), ctypes.byref(gx), ctypes.byref(gy))
    return rc, gx.value, gy.value


def footprint(params: Sequence[seeds_params]) -> int:
    arr = (seeds_params * len(params))(*params)
    out = ctypes.c_int64()
    check(lib.seeds_footprint(arr, len(params), ctypes.byref(out)), "seeds_footprint")
    return out.value


def _ptrs(values, ctype=ctypes.c_void_p):
    return (ctype * len(values))(*values)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def superpixels(images, num_superpixels, block_levels=None, bins_per_channel=5, iters_per_level=2, patch=3,
                gamma=(1, 1), color_space=0, means_iters=0, compactness=0, edge_threshold=0, compact_prior=0,
                stream=None):
    """SEEDS labels for a list of uint8 (H, W, 3) CUDA images in one
    persistent launch: a list of int32 (H, W) CUDA tensors, values in
    [0, K_actual).  `num_superpixels` is one requested K or one per image;
    block_levels=None takes min(4, the most the grid allows) per image.  The
    context is built for this call; reuse a SeedsContext to keep it."""
    import torch
    n = len(images)
    ks = list(num_superpixels) if hasattr(num_superpixels, "__len__") else [num_superpixels] * n
    params = []
    for img, k in zip(images, ks):
        H, W = int(img.shape[0]), int(img.shape[1])
        L = min(4, feasible_levels(W, H, k)) if block_levels is None else block_levels
        params.append(make_params(W, H, k, L, bins_per_channel, iters_per_level, patch, gamma, color_space,
                                  means_iters, compactness, edge_threshold, compact_prior))
    ctx = SeedsContext(params)
    outs = [torch.empty((int(t.shape[0]), int(t.shape[1])), dtype=torch.int32, device=t.device) for t in images]
    ctx.run(images, outs, stream)
    return outs


# --------------------------------------------------------------------------
# autotune cache: tunings in a JSON file keyed by the batch's shapes
# --------------------------------------------------------------------------

_TUNING_FIELDS = [f for f, _ in seeds_tuning._fields_]


def tuning_cache_key(params: Sequence[seeds_params], device: str) -> str:
    """The batch's parameter sets, in order, and the device name, hashed."""
    import hashlib
    import json
    rows = [[getattr(p, f) for f, _ in seeds_params._fields_] for p in params]
    return hashlib.sha256(json.dumps([device, rows]).encode()).hexdigest()[:32]


def load_cached_tuning(path: str, key: str) -> Optional[seeds_tuning]:
    import json
    try:
        with open(path) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    return seeds_tuning(*[int(rec.get(f, 0)) for f in _TUNING_FIELDS])


def store_tuning(path: str, key: str, t: seeds_tuning, note: str = "") -> None:
    import json
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = dict({f: int(getattr(t, f)) for f in _TUNING_FIELDS}, note=note)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class SeedsContext:
    """One library context over a list of image parameter sets.

    Images and label buffers are torch tensors: uint8 (H, W, 3) on the GPU
    (any row stride with unit channel/column strides) and int32 (H, W)."""

    def __init__(self, params: Sequence[seeds_params]):
        self.params = list(params)
        self.n = len(self.params)
        arr = (seeds_params * self.n)(*self.params)
        h = ctypes.c_void_p()
        check(lib.seeds_batch_create(arr, self.n, ctypes.byref(h)), "seeds_batch_create")
        self._h = h
        self.num_superpixels: List[int] = []
        for i in range(self.n):
            k = ctypes.c_int32()
            check(lib.seeds_batch_num_superpixels(self._h, i, ctypes.byref(k)), "seeds_batch_num_superpixels")
            self.num_superpixels.append(k.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.seeds_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling helpers
    @staticmethod
    def _rgb_args(images):
        ptrs, strides = [], []
        for t in images:
            assert t.dtype.itemsize == 1 and t.dim() == 3 and t.shape[2] == 3 and t.is_cuda
            assert t.stride(2) == 1 and t.stride(1) == 3
            ptrs.append(t.data_ptr())
            strides.append(t.stride(0))
        return _ptrs(ptrs), _ptrs(strides, ctypes.c_int64)

    def iterate(self, images, stream=None):
        rgb, strides = self._rgb_args(images)
        check(lib.seeds_batch_iterate(self._h, rgb, strides, _stream_handle(stream)), "seeds_batch_iterate")

    def labels(self, outs, stream=None):
        for t in outs:
            assert t.is_contiguous() and t.is_cuda and t.element_size() == 4
        check(lib.seeds_batch_labels(self._h, _ptrs([t.data_ptr() for t in outs]), _stream_handle(stream)),
              "seeds_batch_labels")

    def run(self, images, outs, stream=None):
        rgb, strides = self._rgb_args(images)
        for t in outs:
            assert t.is_contiguous() and t.is_cuda and t.element_size() == 4
        check(lib.seeds_batch_run(self._h, rgb, strides, _ptrs([t.data_ptr() for t in outs]),
                                  _stream_handle(stream)), "seeds_batch_run")

    def capture(self, images, outs):
        """A CUDA graph of one run over these device buffers: runs once to
        build and cache the schedule, then records the call (a pointer
        upload, a barrier reset and the persistent launch: no allocation, no
        synchronisation) on a side stream.  Refill `images` and call
        graph.replay() to run again."""
        import torch
        self.run(images, outs)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                self.run(images, outs)
        torch.cuda.current_stream().wait_stream(side)
        return graph

    def run_anytime(self, images, outs, max_steps=0, budget_ns=0, stream=None):
        """Anytime termination (Sec. 5.4): run, stopping after max_steps
        steps or budget_ns of device time (0 = no limit); asynchronous, see
        anytime_steps()."""
        rgb, strides = self._rgb_args(images)
        for t in outs:
            assert t.is_contiguous() and t.is_cuda and t.element_size() == 4
        check(lib.seeds_batch_run_anytime(self._h, rgb, strides, _ptrs([t.data_ptr() for t in outs]),
                                          int(max_steps), int(budget_ns), _stream_handle(stream)),
              "seeds_batch_run_anytime")

    def anytime_steps(self) -> int:
        """Steps the last run_anytime launch ran (waits for it)."""
        n = ctypes.c_int32()
        check(lib.seeds_anytime_steps(self._h, ctypes.byref(n)), "seeds_anytime_steps")
        return n.value

    @staticmethod
    def _host_io(images, outs):
        ptrs, strides = [], []
        for t in images:
            assert not t.is_cuda and t.stride(2) == 1 and t.stride(1) == 3
            ptrs.append(t.data_ptr())
            strides.append(t.stride(0))
        for t in outs:
            assert not t.is_cuda and t.is_contiguous() and t.element_size() == 4
        return ptrs, strides, [t.data_ptr() for t in outs]

    def run_host(self, images, outs, stream=None):
        """images: host uint8 (H, W, 3) tensors; outs: host int32 (H, W)."""
        ptrs, strides, optrs = self._host_io(images, outs)
        check(lib.seeds_run_host(self._h, _ptrs(ptrs), _ptrs(strides, ctypes.c_int64), _ptrs(optrs),
                                 _stream_handle(stream)), "seeds_run_host")

    def run_host_stream(self, batches, outs, stream=None):
        """batches[b]: the batch's host uint8 (H, W, 3) tensors; outs[b]: its
        host int32 (H, W) label tensors.  One call for the whole sequence,
        copies of one batch overlapping the launch of another."""
        assert len(batches) == len(outs)
        ptrs, strides, optrs = [], [], []
        for imgs, labs in zip(batches, outs):
            assert len(imgs) == len(labs) == self.n
            p, st, o = self._host_io(imgs, labs)
            ptrs += p
            strides += st
            optrs += o
        check(lib.seeds_run_host_stream(self._h, len(batches), _ptrs(ptrs), _ptrs(strides, ctypes.c_int64),
                                        _ptrs(optrs), _stream_handle(stream)), "seeds_run_host_stream")

    def status(self) -> int:
        return lib.seeds_status(self._h)

    def check_status(self):
        check(self.status(), "seeds_status")

    def set_tuning(self, threads_per_block=0, blocks_per_sm=0, hist_layout=0, small_block_area=0, pixel_tile_rows=0,
                   block_tiles=0):
        t = seeds_tuning(threads_per_block, blocks_per_sm, hist_layout, small_block_area, pixel_tile_rows,
                         block_tiles)
        check(lib.seeds_set_tuning(self._h, ctypes.byref(t)), "seeds_set_tuning")

    def autotune(self, images, outs, reps=3, stream=None, cache: Optional[str] = None) -> seeds_tuning:
        """Time the result-invariant knobs on these inputs and keep the
        fastest.  With `cache` (a JSON file path), a batch of the same
        parameter sets on the same device reuses the stored knobs without
        timing, and a new one is stored after tuning."""
        key = None
        if cache:
            import torch
            key = tuning_cache_key(self.params, torch.cuda.get_device_name())
            hit = load_cached_tuning(cache, key)
            if hit is not None:
                self.set_tuning(*[getattr(hit, f) for f in _TUNING_FIELDS])
                return self.get_tuning()
        rgb, strides = self._rgb_args(images)
        best = seeds_tuning()
        check(lib.seeds_autotune(self._h, rgb, strides, _ptrs([t.data_ptr() for t in outs]), reps,
                                 _stream_handle(stream), ctypes.byref(best)), "seeds_autotune")
        if cache:
            store_tuning(cache, key, best, "%d images, first %dx%d" % (self.n, self.params[0].width,
                                                                       self.params[0].height))
        return best

    def get_tuning(self) -> seeds_tuning:
        t = seeds_tuning()
        check(lib.seeds_get_tuning(self._h, ctypes.byref(t)), "seeds_get_tuning")
        return t

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        check(lib.seeds_debug_launch_count(self._h, ctypes.byref(n)), "seeds_debug_launch_count")
        return n.value

    def profile(self, enable: bool = True):
        check(lib.seeds_profile_enable(self._h, 1 if enable else 0), "seeds_profile_enable")

    def last_kernel_ms(self) -> float:
        ms = ctypes.c_float()
        check(lib.seeds_profile_last_ms(self._h, ctypes.byref(ms)), "seeds_profile_last_ms")
        return ms.value

    def step_stamps(self):
        """ns stamps of the last profiled launch: start, then per step the
        end of its evaluate slot and of its apply slot."""
        import numpy as np
        n = ctypes.c_int32()
        check(lib.seeds_profile_steps(self._h, None, 0, ctypes.byref(n)), "seeds_profile_steps")
        out = np.zeros(n.value, np.int64)
        check(lib.seeds_profile_steps(self._h, out.ctypes.data, n.value, ctypes.byref(n)), "seeds_profile_steps")
        return out

    # -- test hooks
    def num_ops(self, i: int) -> int:
        n = ctypes.c_int32()
        check(lib.seeds_debug_num_ops(self._h, i, ctypes.byref(n)), "seeds_debug_num_ops")
        return n.value

    def op_info(self, i: int, op: int):
        k, l, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib.seeds_debug_op_info(self._h, i, op, ctypes.byref(k), ctypes.byref(l), ctypes.byref(p)),
              "seeds_debug_op_info")
        return k.value, l.value, p.value

    def run_ops(self, images, op_begin: int, op_end: int, stream=None):
        rgb, strides = self._rgb_args(images)
        check(lib.seeds_debug_run_ops(self._h, rgb, strides, op_begin, op_end, _stream_handle(stream)),
              "seeds_debug_run_ops")

    def read_state(self, i: int, level: int, grid_shape, nbins: int, pixels: int):
        import numpy as np
        K = self.num_superpixels[i]
        lab = np.zeros(grid_shape, np.int32)
        hist = np.zeros((K, nbins), np.int32)
        sizes = np.zeros(K, np.int32)
        bins = np.zeros(pixels, np.int32)
        check(lib.seeds_debug_read_state(self._h, i, level, lab.ctypes.data, hist.ctypes.data, sizes.ctypes.data,
                                         bins.ctypes.data), "seeds_debug_read_state")
        return lab, hist, sizes, bins

    def set_labels(self, i: int, level: int, labels):
        import numpy as np
        labels = np.ascontiguousarray(labels, np.int32)
        check(lib.seeds_debug_set_labels(self._h, i, level, labels.ctypes.data), "seeds_debug_set_labels")

    def inject_error(self):
        check(lib.seeds_debug_inject_error(self._h), "seeds_debug_inject_error")

    def barrier_test(self, timeout_ns: int, withhold_step: int = -1):
        """Failure test: barrier time limit and a withheld arrival (see
        seeds_debug_barrier_test); (0, -1) restores normal launches."""
        check(lib.seeds_debug_barrier_test(self._h, int(timeout_ns), int(withhold_step)),
              "seeds_debug_barrier_test")


class Server:
    """Continuous-batching server (seeds_server_*): host images in, host labels out."""

    def __init__(self, arena_bytes, max_slots=64, epoch_steps=8, max_bins_per_channel=8):
        cfg = seeds_server_config(int(arena_bytes), int(max_slots), int(epoch_steps), int(max_bins_per_channel))
        h = ctypes.c_void_p()
        check(lib.seeds_server_create(ctypes.byref(cfg), ctypes.byref(h)), "seeds_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.seeds_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, params: seeds_params, h_rgb, h_labels) -> int:
        """h_rgb: host uint8 (H, W, 3) tensor or array; h_labels: host int32 (H, W)."""
        ptr_rgb, stride = _host_ptr_stride(h_rgb)
        ptr_out, _ = _host_ptr_stride(h_labels)
        rid = ctypes.c_int64()
        check(lib.seeds_server_submit(self._h, ctypes.byref(params), ptr_rgb, stride, ptr_out, ctypes.byref(rid)),
              "seeds_server_submit")
        return rid.value

    def step(self) -> int:
        n = ctypes.c_int32()
        check(lib.seeds_server_step(self._h, ctypes.byref(n)), "seeds_server_step")
        return n.value

    def poll(self, cap=4096):
        ids = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int32()
        check(lib.seeds_server_poll(self._h, ids, ms, cap, ctypes.byref(n)), "seeds_server_poll")
        return [(ids[i], ms[i]) for i in range(n.value)]

    def drain(self):
        check(lib.seeds_server_drain(self._h), "seeds_server_drain")

    def stats(self) -> seeds_server_stats_t:
        st = seeds_server_stats_t()
        check(lib.seeds_server_stats(self._h, ctypes.byref(st)), "seeds_server_stats")
        return st


def _host_ptr_stride(a):
    """(address, row stride in bytes) of a host tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda
        return a.data_ptr(), a.stride(0) * a.element_size()
    return a.ctypes.data, a.strides[0]
