"""Serving driver: a timed request stream through the continuous-batching
server of libseeds.so (seeds_server_*).

The server (native code) owns the device arena, the admission queue and the
epoch launches; this module only releases requests at their arrival times,
calls the server, and turns its completion times into latencies.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import binding, synth


@dataclasses.dataclass
class StreamResult:
    latency_ms: np.ndarray      # per request, completion - scheduled arrival
    makespan_ms: float          # first arrival to last completion
    pixels: int
    labels: List[np.ndarray]    # per request, as returned by the server
    max_resident: int
    epochs: int

    @property
    def mpix_per_s(self) -> float:
        return self.pixels / (self.makespan_ms / 1e3) / 1e6

    def percentile(self, q: float) -> float:
        return float(np.percentile(self.latency_ms, q))


def job_params(job: synth.JobSpec) -> binding.seeds_params:
    """Parameters of a job, its levels clamped to what its grid allows."""
    L = job.levels
    if job.clamp_levels:
        L = min(L, binding.feasible_levels(job.image.width, job.image.height, job.num_superpixels))
    return binding.make_params(job.image.width, job.image.height, job.num_superpixels, L, job.bins_per_channel,
                               job.iters_per_level, job.patch, job.gamma, job.color_space, job.means_iters,
                               job.compactness, job.edge_threshold, job.compact_prior)


def run_stream(requests: Sequence[Tuple[float, synth.JobSpec]], images: Sequence, arena_bytes: int,
               max_slots: int = 64, epoch_steps: int = 8, max_bins_per_channel: int = 8,
               pinned: bool = True, keep_labels: bool = True, prepin: int = 8) -> StreamResult:
    """Serve `requests` (arrival time in s, job) whose host images are
    `images` (uint8 HxWx3, one per request).  Arrivals are released in real
    time on the server's clock.

    Requests that name the same image object share one (pinned) copy of it.
    With keep_labels=False a request's label buffer goes back to a pool of
    its size once the request completes, for a later request to reuse, and
    the result carries no labels; each size's pool starts with up to
    `prepin` buffers made before the first arrival, and grows only when
    more requests of that size are resident at once.  A buffer made during
    the stream pins host memory on the release loop's time (~10 ms for a
    3840x2160 label map), so a backlog that needs new buffers grows while
    they are made.  Pinning a separate copy of every image and
    every label map (tens of GB for a 2 s stream at 2000 req/s) made the
    host stall more and more as it pinned and released them: p99 at 1000
    req/s grew from 8 to 47 ms over three streams, against 8-9 ms with shared
    images and reused label buffers.

    Python's cyclic garbage collector is off while the stream runs (one
    collection first, the previous state restored after): a full collection
    stopped this loop for 35-75 ms, and every request that arrived in that
    window waited for it (p99 at 1000 req/s: 46-85 ms with it, 8-12 ms
    without)."""
    import gc
    import torch  # pinned host buffers

    srv = binding.Server(arena_bytes, max_slots, epoch_steps, max_bins_per_channel)
    shared: Dict[int, object] = {}
    srcs = []
    for img in images:
        if id(img) not in shared:
            t = torch.from_numpy(np.ascontiguousarray(img))
            shared[id(img)] = t.pin_memory() if pinned else t
        srcs.append(shared[id(img)])
    params = [job_params(job) for _, job in requests]
    gc_was_on = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        return _serve(srv, requests, params, srcs, pinned, keep_labels, prepin)
    finally:
        if gc_was_on:
            gc.enable()
        srv.close()


def _serve(srv, requests, params, srcs, pinned, keep_labels, prepin) -> StreamResult:
    """run_stream's loop: release, step, poll until every request is done."""
    import torch

    n = len(requests)
    spare: Dict[Tuple[int, int], List[object]] = {}

    def new_buffer(shape):
        o = torch.empty(shape, dtype=torch.int32)
        return o.pin_memory() if pinned else o

    def label_buffer(job):
        shape = (job.image.height, job.image.width)
        pool = spare.get(shape)
        return pool.pop() if pool else new_buffer(shape)

    if keep_labels:  # every request's buffer exists before the first arrival
        outs: List[object] = [label_buffer(job) for _, job in requests]
    else:
        outs = [None] * n
        count: Dict[Tuple[int, int], int] = {}
        for _, job in requests:
            shape = (job.image.height, job.image.width)
            count[shape] = count.get(shape, 0) + 1
        for shape, c in count.items():
            spare[shape] = [new_buffer(shape) for _ in range(min(c, prepin))]

    start = srv.stats().host_ms
    arrival = np.array([start + 1e3 * a for a, _ in requests])
    id_to_req: Dict[int, int] = {}
    done_ms = np.full(n, np.nan)
    submitted = finished = 0
    max_res = 0
    while finished < n:
        now = srv.stats().host_ms
        while submitted < n and arrival[submitted] <= now:
            if outs[submitted] is None:
                outs[submitted] = label_buffer(requests[submitted][1])
            rid = srv.submit(params[submitted], srcs[submitted], outs[submitted])
            id_to_req[rid] = submitted
            submitted += 1
        resident = srv.step()
        max_res = max(max_res, resident)
        for rid, ms in srv.poll():
            i = id_to_req[rid]
            done_ms[i] = ms
            finished += 1
            if not keep_labels:
                spare.setdefault(tuple(outs[i].shape), []).append(outs[i])
        if resident == 0 and submitted < n and finished == submitted:
            # idle until the next arrival
            wait = (arrival[submitted] - srv.stats().host_ms) / 1e3
            if wait > 0:
                time.sleep(min(wait, 0.002))
    srv.drain()
    st = srv.stats()
    lat = done_ms - arrival
    return StreamResult(latency_ms=lat, makespan_ms=float(np.nanmax(done_ms) - arrival[0]),
                        pixels=sum(job.pixels for _, job in requests),
                        labels=[o.numpy() for o in outs] if keep_labels else [],
                        max_resident=max_res, epochs=int(st.epochs))


def image_pool(sizes: Sequence[Tuple[int, int]], per_size: int, seed: int) -> Dict[Tuple[int, int], List[np.ndarray]]:
    """Seeded Voronoi+noise images (cells = pixels/2000, sigma 8), a few per
    size; serving requests draw their content from this pool."""
    rng = np.random.default_rng(seed)
    pool = {}
    for (W, H) in sizes:
        pool[(W, H)] = [synth.make_image(synth.ImageSpec(W, H, seed=int(rng.integers(0, 2**31)),
                                                         cells=max(1, W * H // 2000), sigma=8.0))
                        for _ in range(per_size)]
    return pool


def stream_images(requests, pool) -> List[np.ndarray]:
    """The pool image each request's seed selects."""
    out = []
    for _, job in requests:
        imgs = pool[(job.image.width, job.image.height)]
        out.append(imgs[job.image.seed % len(imgs)])
    return out
