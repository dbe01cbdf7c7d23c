"""Serving (continuous batching): requests of different sizes arrive while
others run; each one's labels must equal the same request run alone and the
oracle's (integer labels: tolerance 0)."""
import numpy as np
import pytest

import gpu_cases as gc
from paper_1309_3848_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def serve(torch):
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1309_3848_gb300 import serve as s
    return s


def mixed_requests(seed, n, rate):
    rng = np.random.default_rng(seed)
    sizes = [(64, 48), (97, 61), (160, 120), (320, 240), (200, 33)]
    out, t = [], 0.0
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        W, H = sizes[int(rng.integers(0, len(sizes)))]
        K = int(rng.integers(8, max(9, W * H // 150)))
        B = int(rng.choice([3, 5, 8]))
        img = synth.ImageSpec(W, H, seed=int(rng.integers(0, 2**31)), cells=max(2, W * H // 800), sigma=8.0)
        out.append((t, synth.JobSpec(img, K, B, 3, int(rng.integers(1, 3)), clamp_levels=True)))
    return out


def test_served_labels_equal_alone_and_oracle(torch, serve):
    from paper_1309_3848_gb300 import binding
    reqs = mixed_requests(5, 24, rate=2000.0)
    imgs = [synth.make_image(j.image) for _, j in reqs]
    # a small arena and few slots: requests queue, overlap and reuse memory
    import gc as pygc
    assert pygc.isenabled()
    res = serve.run_stream(reqs, imgs, arena_bytes=8 << 20, max_slots=4, epoch_steps=4)
    assert pygc.isenabled()  # the collector, off while the stream runs, is back on
    assert res.max_resident > 1
    assert res.epochs > 1
    want = gc.oracle_many([j for _, j in reqs], imgs)
    for i, ((_, job), img) in enumerate(zip(reqs, imgs)):
        assert gc.first_mismatch(res.labels[i], want[i]) is None, "request %d" % i
        alone, _ = gc.gpu_run(binding, torch, [job], [img])
        assert np.array_equal(alone[0], res.labels[i])
    assert np.all(np.isfinite(res.latency_ms)) and np.all(res.latency_ms >= 0)


def test_arena_bounds_residency(torch, serve):
    from paper_1309_3848_gb300 import binding
    # one 320x240 request's footprint plus a little: only one fits at a time
    job = synth.JobSpec(synth.ImageSpec(320, 240, seed=9, cells=40, sigma=8.0), 300, 5, 3, 1)
    one = binding.footprint([serve.job_params(job)]) + 320 * 240 * 7 + (1 << 16)
    reqs = [(0.0, job)] * 3
    img = synth.make_image(job.image)
    res = serve.run_stream(reqs, [img] * 3, arena_bytes=max(one, 1 << 20), max_slots=8, epoch_steps=64)
    assert res.max_resident == 1
    for lab in res.labels[1:]:
        assert np.array_equal(lab, res.labels[0])


def test_stats_count_the_arena_a_resident_request_holds(torch, serve):
    """While a request is resident its footprint (state, image and label
    staging) is out of the arena's free bytes; after it completes and is
    polled the whole arena is free again."""
    from paper_1309_3848_gb300 import binding
    arena = 64 << 20
    job = synth.JobSpec(synth.ImageSpec(640, 480, seed=3, cells=40, sigma=8.0), 300, 5, 3, 1)
    img = synth.make_image(job.image)
    out = np.zeros((480, 640), np.int32)
    srv = binding.Server(arena, 4, 2, 5)
    try:
        st = srv.stats()
        assert st.arena_free_bytes == arena and st.resident == 0
        srv.submit(serve.job_params(job), img, out)
        assert srv.stats().queued == 1
        assert srv.step() == 1  # admitted, first epoch launched
        st = srv.stats()
        # the image and label staging (7 B/px) plus the state, which the
        # context footprint gives to within its alignment padding
        need = binding.footprint([serve.job_params(job)]) + 640 * 480 * 7
        assert st.resident == 1 and st.queued == 0
        assert 640 * 480 * 7 < arena - st.arena_free_bytes and abs(arena - st.arena_free_bytes - need) <= 4096
        done = []
        while not done:
            srv.step()
            done += srv.poll()
        srv.drain()
        st = srv.stats()
        assert st.resident == 0 and st.arena_free_bytes == arena
    finally:
        srv.close()
    assert gc.first_mismatch(out, gc.oracle_run(job, img)) is None


def test_stream_without_kept_labels_reuses_label_buffers(torch, serve):
    """keep_labels=False (the bench's serving sample): every request still
    completes, label buffers of completed requests go to later requests of
    the same size, and the result carries no labels."""
    reqs = mixed_requests(7, 16, rate=4000.0)
    imgs = [synth.make_image(j.image) for _, j in reqs]
    res = serve.run_stream(reqs, imgs, arena_bytes=16 << 20, max_slots=4, epoch_steps=8, keep_labels=False)
    assert res.labels == []
    assert np.all(np.isfinite(res.latency_ms)) and np.all(res.latency_ms >= 0)
    assert res.pixels == sum(j.pixels for _, j in reqs)


def test_request_too_large_for_the_arena_is_refused(torch, serve):
    from paper_1309_3848_gb300 import binding
    srv = binding.Server(1 << 20, 2, 4, 5)
    job = synth.JobSpec(synth.ImageSpec(640, 480, seed=1, cells=10, sigma=8.0), 100, 5, 2, 1)
    img = np.zeros((480, 640, 3), np.uint8)
    out = np.zeros((480, 640), np.int32)
    with pytest.raises(binding.SeedsError) as e:
        srv.submit(serve.job_params(job), img, out)
    assert e.value.code == binding.SEEDS_ERR_NO_MEMORY
    srv.close()


def test_served_lab_and_means_requests(torch, serve):
    """Requests with LAB bins (Sec. 6.2) and means-based iterations (Sec.
    6.5) served among plain ones: the oracle's labels."""
    import dataclasses
    reqs = mixed_requests(11, 18, rate=3000.0)
    reqs = [(t, dataclasses.replace(j, color_space=i % 2, means_iters=(i % 3), compactness=(0, 7, 30)[i % 3]))
            for i, (t, j) in enumerate(reqs)]
    imgs = [synth.make_image(j.image) for _, j in reqs]
    res = serve.run_stream(reqs, imgs, arena_bytes=8 << 20, max_slots=4, epoch_steps=5)
    want = gc.oracle_many([j for _, j in reqs], imgs)
    for i in range(len(reqs)):
        assert gc.first_mismatch(res.labels[i], want[i]) is None, "request %d" % i


def test_served_labels_at_serving_sizes(torch, serve):
    """The serving workload's sizes (up to 3840x2160, up to 5000
    superpixels, 5 bins per channel, up to 4 levels, 2 iterations) in one
    stream with small requests, in an arena that holds one 4K request at a
    time, so that large and small requests overlap and reuse its space:
    every label map equals the same request alone and the oracle."""
    from paper_1309_3848_gb300 import binding
    shapes = [(320, 240, 300), (3840, 2160, 5000), (640, 480, 900), (1920, 1080, 3000), (481, 321, 200),
              (1280, 720, 2000), (320, 240, 4000), (3840, 2160, 1200), (640, 480, 250), (1920, 1080, 800)]
    reqs, t = [], 0.0
    for i, (W, H, K) in enumerate(shapes):
        t += 0.0001  # all within a millisecond: they queue and share epochs
        img = synth.ImageSpec(W, H, seed=7000 + i, cells=max(1, W * H // 2000), sigma=8.0)
        reqs.append((t, synth.JobSpec(img, K, 5, 4, 2, clamp_levels=True)))
    imgs = gc.make_images([j for _, j in reqs])
    big = binding.footprint([serve.job_params(reqs[1][1])]) + 3840 * 2160 * 7
    res = serve.run_stream(reqs, imgs, arena_bytes=big + (48 << 20), max_slots=6, epoch_steps=8,
                           max_bins_per_channel=5)
    assert res.max_resident > 1
    want = gc.oracle_many([j for _, j in reqs], imgs)
    for i, ((_, job), img) in enumerate(zip(reqs, imgs)):
        assert gc.first_mismatch(res.labels[i], want[i]) is None, "request %d (%dx%d)" % (
            i, job.image.width, job.image.height)
        alone, _ = gc.gpu_run(binding, torch, [job], [img])
        assert np.array_equal(alone[0], res.labels[i])
