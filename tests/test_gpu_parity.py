"""GPU parity: the CUDA path through the C ABI against the oracle, bit for
bit (labels, bins, histograms and sizes are integers: tolerance 0)."""
import dataclasses

import numpy as np
import pytest

import gpu_cases as gc
from oracle import ref
from paper_1309_3848_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def binding(torch):
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1309_3848_gb300 import binding as b
    return b


# --------------------------------------------------------------------------
# op by op: full state after every op of the schedule
# --------------------------------------------------------------------------

STEP_CASES = [
    synth.plain_481()[0],
    synth.JobSpec(synth.ImageSpec(64, 48, seed=5, cells=7, sigma=12.0), 12, 4, 2, 2),
    synth.JobSpec(synth.ImageSpec(97, 61, seed=6, cells=9, sigma=10.0, gradient=True), 30, 8, 3, 2, 3, (2, 1)),
    synth.JobSpec(synth.ImageSpec(50, 37, seed=7, cells=5, sigma=15.0), 20, 3, 0, 3, 0, (1, 1)),
    # five block levels: level 1's superpixels span 16 lattice units per
    # side, so its small-block warps take 8 x 4 blocks of units
    synth.JobSpec(synth.ImageSpec(481, 321, seed=8, cells=12, sigma=8.0, gradient=True), 60, 5, 5, 2),
]


@pytest.mark.parametrize("tiles", [1, 2], ids=["per-unit", "tiled"])
@pytest.mark.parametrize("job", STEP_CASES, ids=["481x321", "64x48", "97x61_B8", "50x37_L0", "481x321_L5"])
def test_state_matches_after_every_op(torch, binding, job, tiles):
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    L = gc.oracle_levels(job)
    assert L == gc.gpu_levels(binding, job)
    r = ref.Ref(W, H, job.num_superpixels, L, job.bins_per_channel, job.iters_per_level, job.patch, job.gamma)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    ctx.set_tuning(block_tiles=tiles)
    d = torch.from_numpy(img).cuda()
    nops = ctx.num_ops(0)
    moved_total = 0
    for op in range(nops - 1):
        kind, level, phase = ctx.op_info(0, op)
        ctx.run_ops([d], op, op + 1)
        ctx.check_status()
        if kind == 0:
            r.init(img)
            show = L
        elif kind == 1:
            moved_total += r.run_phase(level, phase)
            show = level
        elif kind == 2:
            show = level - 1
        nbx, nby, _, _ = r.level_grid(show)
        lab, hist, sizes, bins = ctx.read_state(0, show, (nby, nbx), r.nbins, W * H)
        want_lab = r.level_labels(show)
        msg = gc.first_mismatch(lab, want_lab)
        assert msg is None, "op %d (kind %d level %d phase %d): %s" % (op, kind, level, phase, msg)
        h, s = r.hist()
        assert np.array_equal(hist, h), "op %d histograms differ" % op
        assert np.array_equal(sizes, s), "op %d sizes differ" % op
        if kind == 0:
            assert np.array_equal(bins.reshape(H, W), r.bins())
    assert moved_total > 0


@pytest.mark.parametrize("tuning", [dict(small_block_area=1), dict(small_block_area=16, hist_layout=1),
                                    dict(pixel_tile_rows=2), dict(block_tiles=2),
                                    dict(block_tiles=2, pixel_tile_rows=2, small_block_area=4, hist_layout=1),
                                    dict(block_tiles=2, small_block_area=1)])
def test_mixed_bin_batch_matches_after_every_op(torch, binding, tuning):
    """Images with different bin counts (and so different scratch use) in
    one batch, every block judged by a warp or by a thread: full state of
    every image after every op."""
    jobs = [synth.JobSpec(synth.ImageSpec(96, 64, seed=21, cells=8, sigma=12.0), 24, 8, 2, 2),
            synth.JobSpec(synth.ImageSpec(80, 72, seed=22, cells=9, sigma=14.0), 20, 5, 2, 2),
            synth.JobSpec(synth.ImageSpec(64, 64, seed=23, cells=6, sigma=10.0), 16, 3, 2, 2)]
    imgs = [synth.make_image(j.image) for j in jobs]
    refs = [ref.Ref(j.image.width, j.image.height, j.num_superpixels, 2, j.bins_per_channel, 2) for j in jobs]
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    ctx.set_tuning(**tuning)
    d = [torch.from_numpy(im).cuda() for im in imgs]
    nops = ctx.num_ops(0)
    assert all(ctx.num_ops(i) == nops for i in range(len(jobs)))
    for op in range(nops - 1):
        kind, level, phase = ctx.op_info(0, op)
        ctx.run_ops(d, op, op + 1)
        ctx.check_status()
        for i, (j, r, im) in enumerate(zip(jobs, refs, imgs)):
            if kind == 0:
                r.init(im)
                show = 2
            elif kind == 1:
                r.run_phase(level, phase)
                show = level
            else:
                show = level - 1
            nbx, nby, _, _ = r.level_grid(show)
            lab, hist, sizes, _ = ctx.read_state(i, show, (nby, nbx), r.nbins, j.pixels)
            assert gc.first_mismatch(lab, r.level_labels(show)) is None, "image %d op %d" % (i, op)
            h, s = r.hist()
            assert np.array_equal(hist, h) and np.array_equal(sizes, s), "image %d op %d" % (i, op)


# --------------------------------------------------------------------------
# a single phase from injected (non-grid) states
# --------------------------------------------------------------------------

def test_single_phases_from_injected_states(torch, binding):
    rng = np.random.default_rng(3)
    job = synth.JobSpec(synth.ImageSpec(80, 60, seed=8, cells=10, sigma=14.0), 24, 5, 2, 3)
    W, H = 80, 60
    img = synth.make_image(job.image)
    d = torch.from_numpy(img).cuda()
    r = ref.Ref(W, H, 24, 2, 5, 3)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    ctx.run_ops([d], 0, 1)  # bins
    # states reached by the oracle's own sequential mode: ragged but valid
    _, _, _ = r.sequential(img, seed=int(rng.integers(0, 1 << 30)))
    state = r.labels()
    ops = [(op,) + ctx.op_info(0, op) for op in range(ctx.num_ops(0))]
    pixel_ops = [o for o in ops if o[1] == 1 and o[2] == 0]
    for op, kind, level, phase in pixel_ops[:4]:
        r.set_labels(state)
        ctx.set_labels(0, 0, state)
        ctx.run_ops([d], op, op + 1)
        ctx.check_status()
        r.run_phase(0, phase)
        lab, hist, sizes, _ = ctx.read_state(0, 0, (H, W), r.nbins, W * H)
        assert gc.first_mismatch(lab, r.labels()) is None
        h, s = r.hist()
        assert np.array_equal(hist, h) and np.array_equal(sizes, s)


# --------------------------------------------------------------------------
# whole schedule on the workloads
# --------------------------------------------------------------------------

def check_jobs(torch, binding, jobs, tuning=None):
    imgs = gc.make_images(jobs)
    got, ctx = gc.gpu_run(binding, torch, jobs, imgs, tuning)
    want = gc.oracle_many(jobs, imgs)
    for i, (a, b) in enumerate(zip(got, want)):
        msg = gc.first_mismatch(a, b)
        assert msg is None, "image %d (%dx%d): %s" % (i, jobs[i].image.width, jobs[i].image.height, msg)
    return got


def test_plain_481x321(torch, binding):
    check_jobs(torch, binding, synth.plain_481())


def test_plain_1920x1080(torch, binding):
    check_jobs(torch, binding, synth.plain_1080())


def test_batch64_mixed(torch, binding):
    check_jobs(torch, binding, synth.batch_64())


def test_batch16_3840x2160(torch, binding):
    check_jobs(torch, binding, synth.batch_4k())


@pytest.mark.parametrize("seed", range(4))
def test_random_small_jobs(torch, binding, seed):
    jobs = synth.random_small_jobs(1000 + seed, 24, max_side=96)
    for j in jobs:
        assert gc.oracle_levels(j) == gc.gpu_levels(binding, j)
    # one batch of mixed parameters, and each image alone
    got = check_jobs(torch, binding, jobs)
    for i in range(0, len(jobs), 6):
        alone, _ = gc.gpu_run(binding, torch, [jobs[i]], [synth.make_image(jobs[i].image)])
        assert np.array_equal(alone[0], got[i])


def test_edge_sizes(torch, binding):
    jobs = [
        synth.JobSpec(synth.ImageSpec(1, 1, seed=1, cells=1, sigma=0.0), 1, 5, 0, 2),
        synth.JobSpec(synth.ImageSpec(1, 40, seed=2, cells=3, sigma=9.0), 4, 5, 0, 2),
        synth.JobSpec(synth.ImageSpec(40, 1, seed=3, cells=3, sigma=9.0), 4, 5, 0, 2),
        synth.JobSpec(synth.ImageSpec(2, 2, seed=4, cells=2, sigma=30.0), 4, 2, 0, 3),
        synth.JobSpec(synth.ImageSpec(33, 17, seed=5, cells=4, sigma=20.0), 1, 4, 4, 2),
        synth.JobSpec(synth.ImageSpec(64, 64, seed=6, cells=6, sigma=20.0), 4, 16, 4, 2),  # 4096 bins
        synth.JobSpec(synth.ImageSpec(31, 29, seed=7, cells=5, sigma=20.0), 900, 3, 0, 2),  # ~1 px superpixels
    ]
    check_jobs(torch, binding, jobs)


# --------------------------------------------------------------------------
# result-invariant knobs and call forms
# --------------------------------------------------------------------------

TUNINGS = [dict(threads_per_block=128), dict(threads_per_block=512, hist_layout=1),
           dict(hist_layout=1, small_block_area=1), dict(blocks_per_sm=1, small_block_area=4),
           dict(threads_per_block=256, blocks_per_sm=2, hist_layout=0, small_block_area=9),
           dict(pixel_tile_rows=2), dict(threads_per_block=512, pixel_tile_rows=2, small_block_area=1),
           dict(block_tiles=2), dict(block_tiles=2, small_block_area=4, pixel_tile_rows=2),
           dict(block_tiles=1, threads_per_block=256), dict(block_tiles=2, small_block_area=1, blocks_per_sm=1)]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_tuning_does_not_change_labels(torch, binding, tuning):
    jobs = synth.plain_481() + synth.random_small_jobs(77, 6, max_side=80)
    check_jobs(torch, binding, jobs, tuning)


def test_iterate_then_labels_and_host_path(torch, binding):
    job = synth.plain_481()[0]
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    want = gc.oracle_run(job, img)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    out = torch.empty((H, W), dtype=torch.int32, device="cuda")
    for _ in range(2):  # the context re-initialises from the image every call
        ctx.iterate([d])
        ctx.labels([out])
        ctx.check_status()
        assert np.array_equal(out.cpu().numpy(), want)
    # from host memory, pinned and pageable; padded rows
    pad = np.zeros((H, W * 3 + 17), np.uint8)
    pad[:, :W * 3] = img.reshape(H, W * 3)
    host_img = torch.from_numpy(pad)[:, :W * 3].reshape(H, W, 3)
    assert host_img.stride(0) == W * 3 + 17
    for pinned in (False, True):
        src = host_img.pin_memory() if pinned else host_img
        dst = torch.empty((H, W), dtype=torch.int32)
        dst = dst.pin_memory() if pinned else dst
        ctx.run_host([src], [dst])
        torch.cuda.synchronize()
        ctx.check_status()
        assert np.array_equal(dst.numpy(), want)


def test_streamed_host_runs_match_the_oracle_batch_by_batch(torch, binding):
    """seeds_run_host_stream: five batches of two images (three distinct
    image sets, one of them pageable with padded rows), copies overlapping
    the launches through two staging slots; every batch's labels equal the
    oracle's, and host runs before and after on the same context still do."""
    jobs = [synth.JobSpec(synth.ImageSpec(97, 61, seed=6, cells=9, sigma=10.0, gradient=True), 30, 8, 3, 2, 3),
            synth.JobSpec(synth.ImageSpec(64, 48, seed=5, cells=7, sigma=12.0), 12, 4, 2, 2)]
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    sets, wants = [], []
    for s in range(3):
        imgs = [synth.make_image(dataclasses.replace(j.image, seed=j.image.seed + 10 * s)) for j in jobs]
        wants.append([gc.oracle_run(j, im) for j, im in zip(jobs, imgs)])
        if s == 2:  # pageable, rows 5 bytes apart beyond 3*W
            host = []
            for im in imgs:
                H, W = im.shape[:2]
                pad = np.zeros((H, W * 3 + 5), np.uint8)
                pad[:, :W * 3] = im.reshape(H, W * 3)
                host.append(torch.from_numpy(pad)[:, :W * 3].reshape(H, W, 3))
        else:
            host = [torch.from_numpy(im).pin_memory() for im in imgs]
        sets.append(host)
    order = [0, 1, 2, 0, 1]
    outs = [[torch.full((j.image.height, j.image.width), -1, dtype=torch.int32).pin_memory() for j in jobs]
            for _ in order]
    single = [torch.empty((j.image.height, j.image.width), dtype=torch.int32).pin_memory() for j in jobs]
    ctx.run_host(sets[1], single)
    ctx.run_host_stream([sets[s] for s in order], outs)
    ctx.run_host(sets[2], single)
    torch.cuda.synchronize()
    ctx.check_status()
    for s, o in zip(order, outs):
        for w, t in zip(wants[s], o):
            assert np.array_equal(t.numpy(), w)
    for w, t in zip(wants[2], single):
        assert np.array_equal(t.numpy(), w)
    one = [torch.empty_like(t) for t in outs[0]]  # a stream of one batch
    ctx.run_host_stream([sets[1]], [one])
    torch.cuda.synchronize()
    for w, t in zip(wants[1], one):
        assert np.array_equal(t.numpy(), w)
    bad = binding.lib.seeds_run_host_stream(ctx._h, 0, None, None, None, None)
    assert bad == binding.SEEDS_ERR_INVALID


def test_strided_device_image(torch, binding):
    job = synth.plain_481()[0]
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    big = torch.zeros((H, W + 5, 3), dtype=torch.uint8, device="cuda")
    big[:, :W] = torch.from_numpy(img).cuda()
    view = big[:, :W]
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    out = torch.empty((H, W), dtype=torch.int32, device="cuda")
    ctx.run([view], [out])
    ctx.check_status()
    assert np.array_equal(out.cpu().numpy(), gc.oracle_run(job, img))


def test_streams_give_identical_labels(torch, binding):
    jobs = synth.random_small_jobs(5, 4, max_side=120)
    imgs = gc.make_images(jobs)
    want = gc.oracle_many(jobs, imgs)
    s = torch.cuda.Stream()
    ctxs = [binding.SeedsContext([gc.params_for(binding, j)]) for j in jobs]
    outs = []
    with torch.cuda.stream(s):
        for ctx, j, im in zip(ctxs, jobs, imgs):
            o = torch.empty((j.image.height, j.image.width), dtype=torch.int32, device="cuda")
            ctx.run([torch.from_numpy(im).cuda()], [o], stream=s)
            outs.append(o)
    s.synchronize()
    for ctx, o, w in zip(ctxs, outs, want):
        ctx.check_status()
        assert np.array_equal(o.cpu().numpy(), w)


# --------------------------------------------------------------------------
# failure reporting (host-side injection; no GPU fault)
# --------------------------------------------------------------------------

def test_device_error_word_is_reported_and_cleared(torch, binding):
    job = synth.plain_481()[0]
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    ctx.inject_error()
    assert ctx.status() == binding.SEEDS_ERR_DEVICE
    assert ctx.status() == binding.SEEDS_OK
    img = synth.make_image(job.image)
    out = torch.empty((job.image.height, job.image.width), dtype=torch.int32, device="cuda")
    ctx.run([torch.from_numpy(img).cuda()], [out])
    ctx.check_status()
    assert np.array_equal(out.cpu().numpy(), gc.oracle_run(job, img))


@pytest.mark.parametrize("anytime", [False, True], ids=["counting_barrier", "stop_barrier"])
def test_barrier_wait_that_runs_out_is_reported_and_the_context_recovers(torch, binding, anytime):
    """A bounded device-side wait made to run out (CTA 0 withholds its
    arrival at one barrier; the limit is 0.2 ms): every CTA gives up, sets
    the error word and leaves the kernel, no label is written, the status
    reads SEEDS_ERR_DEVICE, and the next normal run on the same context
    gives the oracle's labels."""
    job = synth.plain_481()[0]
    img = synth.make_image(job.image)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    for step in (0, 5, ctx.num_ops(0) - 2):
        ctx.barrier_test(200_000, step)
        out.fill_(-1)
        if anytime:
            ctx.run_anytime([d], [out])
        else:
            ctx.run([d], [out])
        torch.cuda.synchronize()
        assert ctx.status() == binding.SEEDS_ERR_DEVICE, step
        assert ctx.status() == binding.SEEDS_OK
        assert int((out != -1).sum()) == 0, "labels written after the wait ran out at step %d" % step
    ctx.barrier_test(0, -1)
    ctx.run([d], [out])
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(out.cpu().numpy(), gc.oracle_run(job, img))


def test_launch_count(torch, binding):
    job = synth.plain_481()[0]
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    img = torch.from_numpy(synth.make_image(job.image)).cuda()
    out = torch.empty((job.image.height, job.image.width), dtype=torch.int32, device="cuda")
    n0 = ctx.launch_count()
    ctx.run([img], [out])
    ctx.check_status()
    assert ctx.launch_count() - n0 == 2  # pointer upload + one persistent kernel


def test_autotune_keeps_labels(torch, binding):
    jobs = synth.plain_481() + synth.random_small_jobs(31, 5, max_side=120)
    imgs = gc.make_images(jobs)
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty((j.image.height, j.image.width), dtype=torch.int32, device="cuda") for j in jobs]
    best = ctx.autotune(d, outs, reps=2)
    assert best.threads_per_block in (128, 256, 512, 1024)
    t = ctx.get_tuning()
    assert (t.threads_per_block, t.blocks_per_sm, t.hist_layout, t.small_block_area, t.pixel_tile_rows) == \
        (best.threads_per_block, best.blocks_per_sm, best.hist_layout, best.small_block_area, best.pixel_tile_rows)
    for o in outs:
        o.fill_(-1)
    ctx.run(d, outs)
    ctx.check_status()
    want = gc.oracle_many(jobs, imgs)
    for o, w in zip(outs, want):
        assert np.array_equal(o.cpu().numpy(), w)


def test_set_tuning_that_cannot_launch_leaves_context_usable(torch, binding):
    # 4096 bins: 512-thread blocks need more shared memory than a block may have
    job = synth.JobSpec(synth.ImageSpec(64, 64, seed=6, cells=6, sigma=20.0), 4, 16, 2, 2)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    before = ctx.get_tuning()
    with pytest.raises(binding.SeedsError):
        ctx.set_tuning(threads_per_block=512)
    after = ctx.get_tuning()
    assert after.threads_per_block == before.threads_per_block
    got, _ = gc.gpu_run(binding, torch, [job], [synth.make_image(job.image)])
    assert np.array_equal(got[0], gc.oracle_run(job, synth.make_image(job.image)))


def test_autotune_cache_reuses_the_knobs(torch, binding, tmp_path):
    jobs = synth.random_small_jobs(33, 4, max_side=100)
    imgs = gc.make_images(jobs)
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty((j.image.height, j.image.width), dtype=torch.int32, device="cuda") for j in jobs]
    path = str(tmp_path / "tunings.json")
    first = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    t1 = first.autotune(d, outs, reps=1, cache=path)
    second = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    n0 = second.launch_count()
    t2 = second.autotune(d, outs, reps=1, cache=path)
    assert second.launch_count() == n0  # a cache hit times nothing
    fields = ("threads_per_block", "blocks_per_sm", "hist_layout", "small_block_area", "pixel_tile_rows")
    assert [getattr(t1, f) for f in fields] == [getattr(t2, f) for f in fields]
    second.run(d, outs)
    torch.cuda.synchronize()
    second.check_status()
    for o, w in zip(outs, gc.oracle_many(jobs, imgs)):
        assert gc.first_mismatch(o.cpu().numpy(), w) is None


def test_contexts_of_different_bin_counts_interleave(torch, binding):
    """The kernel's shared-memory limit is one setting per device: a context
    made for 512 bins still launches after a 125-bin context and the
    allocation-free entry point configured theirs, with the oracle's labels."""
    import ctypes
    big = synth.JobSpec(synth.ImageSpec(160, 120, seed=71, cells=30, sigma=6.0), 120, 8, 3, 2)
    small = synth.JobSpec(synth.ImageSpec(120, 90, seed=72, cells=20, sigma=6.0), 60, 5, 2, 2)
    imgs = [synth.make_image(big.image), synth.make_image(small.image)]
    want = gc.oracle_many([big, small], imgs)
    c_big = binding.SeedsContext([gc.params_for(binding, big)])
    c_small = binding.SeedsContext([gc.params_for(binding, small)])
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full((j.image.height, j.image.width), -1, dtype=torch.int32, device="cuda") for j in (big, small)]
    p = gc.params_for(binding, small)
    rc = binding.lib.seeds_run_static(ctypes.byref(p), d[1].data_ptr(), d[1].stride(0), outs[1].data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == binding.SEEDS_OK
    for _ in range(2):
        c_big.run([d[0]], [outs[0]])
        c_small.run([d[1]], [outs[1]])
    torch.cuda.synchronize()
    c_big.check_status()
    c_small.check_status()
    for o, w in zip(outs, want):
        assert gc.first_mismatch(o.cpu().numpy(), w) is None
