"""GPU parity of edge snapping (the edge prior of Sec. 6.4, reading R18): the
state after every op, whole runs in RGB and LAB, with and without the means
iterations, mixed batches and the allocation-free entry point, bit for bit
against the oracle."""
import ctypes
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


def edges(job, tau, color=0, means=0, m=0):
    return dataclasses.replace(job, edge_threshold=tau, color_space=color, means_iters=means, compactness=m)


def oracle_ref(job):
    return ref.Ref(job.image.width, job.image.height, job.num_superpixels, gc.oracle_levels(job),
                   job.bins_per_channel, job.iters_per_level, job.patch, job.gamma, job.color_space,
                   job.means_iters, job.compactness, job.edge_threshold)


STEP_CASES = [
    edges(synth.plain_481()[0], 60),
    edges(synth.JobSpec(synth.ImageSpec(97, 61, seed=16, cells=9, sigma=10.0, gradient=True), 30, 8, 3, 1, 3, (2, 1)),
          25, 1, 2, 10),
    edges(synth.JobSpec(synth.ImageSpec(50, 37, seed=17, cells=5, sigma=15.0), 20, 3, 0, 2, 0, (1, 1)), 1),
]


@pytest.mark.parametrize("job", STEP_CASES, ids=["481x321_tau60", "97x61_lab_means_tau25", "50x37_L0_tau1"])
def test_state_matches_after_every_op(torch, binding, job):
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    L = gc.oracle_levels(job)
    r = oracle_ref(job)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    nops = ctx.num_ops(0)
    assert nops == r.num_ops()
    for op in range(nops - 1):
        kind, level, phase = ctx.op_info(0, op)
        ctx.run_ops([d], op, op + 1)
        ctx.check_status()
        if kind == 0:
            r.init(img)
            show = L
        elif kind == 1:
            r.run_phase(level, phase)
            show = level
        elif kind == 2:
            show = level - 1
        elif kind == 5:
            show = 0
        else:
            assert kind == 6
            r.run_means_phase(phase)
            show = 0
        nbx, nby, _, _ = r.level_grid(show)
        lab, hist, sizes, _ = ctx.read_state(0, show, (nby, nbx), r.nbins, W * H)
        msg = gc.first_mismatch(lab, r.level_labels(show))
        assert msg is None, "op %d (kind %d level %d phase %d): %s" % (op, kind, level, phase, msg)
        h, s = r.hist()
        assert np.array_equal(hist, h), "op %d histograms differ" % op
        assert np.array_equal(sizes, s), "op %d sizes differ" % op


def check(torch, binding, jobs, tuning=None):
    imgs = gc.make_images(jobs)
    got, _ = gc.gpu_run(binding, torch, jobs, imgs, tuning)
    want = gc.oracle_many(jobs, imgs)
    for i, (a, b) in enumerate(zip(got, want)):
        msg = gc.first_mismatch(a, b)
        assert msg is None, "image %d (%dx%d, tau %d, colour %d, means %d): %s" % (
            i, jobs[i].image.width, jobs[i].image.height, jobs[i].edge_threshold, jobs[i].color_space,
            jobs[i].means_iters, msg)
    return got, want


def test_snapping_changes_the_labels(torch, binding):
    """A threshold inside the image's colour range changes the result, and the
    GPU follows the oracle both ways."""
    job = synth.plain_481()[0]
    got, _ = check(torch, binding, [job, edges(job, 40)])
    assert not np.array_equal(got[0], got[1])


@pytest.mark.parametrize("tau", [1, 30, 90, 765])
def test_plain_481x321_thresholds(torch, binding, tau):
    check(torch, binding, [edges(synth.plain_481()[0], tau)])


def test_plain_1920x1080_lab_with_means(torch, binding):
    check(torch, binding, [edges(synth.plain_1080()[0], 35, 1, 2, 10)])


def test_batch_mixing_thresholds(torch, binding):
    jobs = synth.random_small_jobs(93, 24, max_side=220)
    jobs = [edges(j, (0, 1, 20, 60)[i % 4], i % 2, (0, 0, 1, 2)[i % 4], (0, 0, 8, 30)[i % 4])
            for i, j in enumerate(jobs)]
    check(torch, binding, jobs)


def test_short_pixel_tiles(torch, binding):
    job = synth.JobSpec(synth.ImageSpec(200, 90, seed=18, cells=20, sigma=9.0), 40, 4, 2, 2)
    check(torch, binding, [edges(synth.plain_481()[0], 45), edges(job, 15, 1, 1, 0)], dict(pixel_tile_rows=2))


def test_anytime_stops_with_snapping(torch, binding):
    job = edges(synth.plain_481()[0], 50, 0, 1, 6)
    img = synth.make_image(job.image)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    nops = oracle_ref(job).num_ops()
    for m in (1, nops // 2, nops - 3, nops):
        ctx.run_anytime([d], [out], max_steps=m)
        steps = ctx.anytime_steps()
        torch.cuda.synchronize()
        ctx.check_status()
        assert steps == m
        msg = gc.first_mismatch(out.cpu().numpy(), oracle_ref(job).run_ops(img, m))
        assert msg is None, "stop after %d steps: %s" % (m, msg)


def test_static_entry_with_snapping(torch, binding):
    job = edges(synth.plain_481()[0], 40, 1)
    img = synth.make_image(job.image)
    d = torch.from_numpy(img).cuda()
    p = gc.params_for(binding, job)
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = binding.lib.seeds_run_static(ctypes.byref(p), d.data_ptr(), d.stride(0), out.data_ptr(),
                                      status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == binding.SEEDS_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert gc.first_mismatch(out.cpu().numpy(), gc.oracle_run(job, img)) is None
