"""Host logic of the serving driver (serve.run_stream) on the CPU, against a
fake server that finishes each request three steps after its admission:
every request is served once, in order, with latencies on the server's
clock; requests naming one image share one source buffer; label buffers go
to later requests only when labels are not kept, and never to two resident
requests at once; the garbage collector is off during the stream and its
previous state comes back."""
import gc
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1309_3848_gb300 import binding, serve, synth


class FakeServer:
    last = None

    def __init__(self, arena_bytes, max_slots=64, epoch_steps=8, max_bins_per_channel=8):
        self.t0 = time.perf_counter()
        self.next_id = 0
        self.live = {}      # id -> [steps left, label buffer]
        self.finished = []  # (id, ms) not yet polled
        self.epochs = 0
        self.srcs, self.outs, self.gc_on = [], [], []
        self.closed = False
        FakeServer.last = self

    def stats(self):
        return SimpleNamespace(host_ms=(time.perf_counter() - self.t0) * 1e3, epochs=self.epochs, queued=0,
                               resident=len(self.live))

    def submit(self, params, src, out):
        assert all(o is not out for _, o in self.live.values()), "a label buffer given to two resident requests"
        rid = self.next_id
        self.next_id += 1
        self.live[rid] = [3, out]
        self.srcs.append(src)
        self.outs.append(out)
        self.gc_on.append(gc.isenabled())
        return rid

    def step(self):
        n = len(self.live)
        if n:
            self.epochs += 1
        for rid in list(self.live):
            self.live[rid][0] -= 1
            if self.live[rid][0] == 0:
                self.live.pop(rid)[1].fill_(rid)
                self.finished.append((rid, self.stats().host_ms))
        return n

    def poll(self):
        out, self.finished = self.finished, []
        return out

    def drain(self):
        assert not self.live

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(binding, "Server", FakeServer)
    return FakeServer


def stream(n=24, gap_s=0.0005):
    sizes = [(64, 48), (97, 61), (50, 37)]
    pool = serve.image_pool(sizes, 2, seed=3)
    reqs = []
    for i in range(n):
        W, H = sizes[i % 3]
        img = synth.ImageSpec(W, H, seed=i // 3, cells=4, sigma=8.0)
        reqs.append((i * gap_s, synth.JobSpec(img, 12, 5, 1, 1, clamp_levels=True)))
    return reqs, serve.stream_images(reqs, pool)


def test_every_request_is_served_once_with_its_own_labels(fake):
    reqs, imgs = stream()
    res = serve.run_stream(reqs, imgs, arena_bytes=1 << 20, pinned=False)
    srv = fake.last
    assert srv.closed and srv.next_id == len(reqs)
    assert len(res.labels) == len(reqs)
    for i, lab in enumerate(res.labels):  # request i was submitted i-th: the fake wrote its id
        assert lab.shape == (reqs[i][1].image.height, reqs[i][1].image.width) and np.all(lab == i)
    assert len({id(o) for o in srv.outs}) == len(reqs)
    assert len({id(s) for s in srv.srcs}) == len({id(im) for im in imgs}) < len(reqs)
    assert np.all(np.isfinite(res.latency_ms)) and np.all(res.latency_ms >= 0)
    assert res.pixels == sum(j.pixels for _, j in reqs) and res.max_resident >= 1


def test_label_buffers_are_reused_only_without_kept_labels(fake):
    reqs, imgs = stream(n=30, gap_s=0.002)
    res = serve.run_stream(reqs, imgs, arena_bytes=1 << 20, pinned=False, keep_labels=False)
    srv = fake.last
    assert res.labels == []
    assert srv.next_id == len(reqs) and np.all(np.isfinite(res.latency_ms))
    # spaced arrivals finish before later ones start: far fewer buffers than requests
    assert len({id(o) for o in srv.outs}) < len(reqs)
    for o, (_, job) in zip(srv.outs, reqs):
        assert tuple(o.shape) == (job.image.height, job.image.width)


@pytest.mark.parametrize("was_on", [True, False])
def test_garbage_collector_is_off_during_the_stream_and_restored(fake, was_on):
    reqs, imgs = stream(n=6)
    if not was_on:
        gc.disable()
    try:
        serve.run_stream(reqs, imgs, arena_bytes=1 << 20, pinned=False)
        assert gc.isenabled() == was_on
        assert fake.last.gc_on == [False] * len(reqs)
    finally:
        gc.enable()


@pytest.mark.parametrize("prepin", [0, 8])
def test_label_pools_are_made_before_the_first_arrival(fake, monkeypatch, prepin):
    """Without kept labels each size's pool is filled before the stream
    starts (up to `prepin` buffers), so no buffer is made on the release
    loop's time while no more than that many requests of a size are
    resident; with prepin=0 they are made as requests arrive."""
    import torch
    made_at = []  # submits done when each label buffer was made
    real_empty = torch.empty

    def counting_empty(*a, **k):
        t = real_empty(*a, **k)
        if k.get("dtype") is torch.int32:
            made_at.append(len(FakeServer.last.srcs))
        return t

    monkeypatch.setattr(torch, "empty", counting_empty)
    reqs, imgs = stream(n=30, gap_s=0.002)
    serve.run_stream(reqs, imgs, arena_bytes=1 << 20, pinned=False, keep_labels=False, prepin=prepin)
    assert made_at
    if prepin:
        assert max(made_at) == 0 and len(made_at) == 3 * min(10, prepin)
    else:
        assert max(made_at) > 0 and len(made_at) < len(reqs)
