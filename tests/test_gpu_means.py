"""GPU parity of the means-based pixel iterations (SPM, Sec. 6.3, run as the
last pixel iterations, Sec. 6.5; reading R17): state after every op, whole
runs, anytime stops inside them and the allocation-free entry point, bit for
bit against the oracle."""
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


def means(job, iters=2, m=0, color=0):
    return dataclasses.replace(job, means_iters=iters, compactness=m, color_space=color)


def oracle_ref(job):
    return ref.Ref(job.image.width, job.image.height, job.num_superpixels, gc.oracle_levels(job),
                   job.bins_per_channel, job.iters_per_level, job.patch, job.gamma, job.color_space,
                   job.means_iters, job.compactness, job.edge_threshold)


STEP_CASES = [
    means(synth.plain_481()[0], 2, 0),
    means(synth.JobSpec(synth.ImageSpec(97, 61, seed=6, cells=9, sigma=10.0, gradient=True), 30, 8, 3, 1, 3, (2, 1)),
          2, 20, 1),
    means(synth.JobSpec(synth.ImageSpec(50, 37, seed=7, cells=5, sigma=15.0), 20, 3, 0, 1, 0, (1, 1)), 3, 5),
]


@pytest.mark.parametrize("job", STEP_CASES, ids=["481x321_m0", "97x61_lab_m20", "50x37_L0_m5"])
def test_state_matches_after_every_op(torch, binding, job):
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    L = gc.oracle_levels(job)
    r = oracle_ref(job)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    nops = ctx.num_ops(0)
    assert nops == r.num_ops()
    moved = 0
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
            moved += r.run_means_phase(phase)
            show = 0
        nbx, nby, _, _ = r.level_grid(show)
        lab, hist, sizes, _ = ctx.read_state(0, show, (nby, nbx), r.nbins, W * H)
        msg = gc.first_mismatch(lab, r.level_labels(show))
        assert msg is None, "op %d (kind %d level %d phase %d): %s" % (op, kind, level, phase, msg)
        h, s = r.hist()
        assert np.array_equal(hist, h), "op %d histograms differ" % op
        assert np.array_equal(sizes, s), "op %d sizes differ" % op
    assert moved > 0, "the means iterations moved nothing"


def check(torch, binding, jobs):
    imgs = gc.make_images(jobs)
    got, _ = gc.gpu_run(binding, torch, jobs, imgs)
    for i, (a, b) in enumerate(zip(got, gc.oracle_many(jobs, imgs))):
        msg = gc.first_mismatch(a, b)
        assert msg is None, "image %d (%dx%d, means %d, m %d): %s" % (
            i, jobs[i].image.width, jobs[i].image.height, jobs[i].means_iters, jobs[i].compactness, msg)


def test_plain_1920x1080_with_means(torch, binding):
    check(torch, binding, [means(synth.plain_1080()[0], 2, 10)])


def test_batch_mixing_means_and_histogram_only_images(torch, binding):
    jobs = synth.random_small_jobs(91, 24, max_side=220)
    jobs = [means(j, 1 + i % 3, (0, 4, 40)[i % 3], i % 2) if i % 4 != 3 else j for i, j in enumerate(jobs)]
    check(torch, binding, jobs)


def test_means_with_short_pixel_tiles(torch, binding):
    small = synth.JobSpec(synth.ImageSpec(200, 90, seed=8, cells=20, sigma=9.0), 40, 4, 2, 2)
    jobs = [means(synth.plain_481()[0], 2, 6), means(small, 1, 0, 1)]
    imgs = gc.make_images(jobs)
    got, _ = gc.gpu_run(binding, torch, jobs, imgs, dict(pixel_tile_rows=2))
    for i, (a, b) in enumerate(zip(got, gc.oracle_many(jobs, imgs))):
        assert gc.first_mismatch(a, b) is None, "image %d" % i


def test_anytime_stops_inside_the_means_iterations(torch, binding):
    job = means(synth.plain_481()[0], 2, 8)
    img = synth.make_image(job.image)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    nops = oracle_ref(job).num_ops()
    for m in range(nops - 11, nops + 1):  # the last pixel phases, the means start, the means phases
        ctx.run_anytime([d], [out], max_steps=m)
        steps = ctx.anytime_steps()
        torch.cuda.synchronize()
        ctx.check_status()
        assert steps == m
        msg = gc.first_mismatch(out.cpu().numpy(), oracle_ref(job).run_ops(img, m))
        assert msg is None, "stop after %d steps: %s" % (m, msg)


def test_static_entry_with_means(torch, binding):
    job = means(synth.plain_481()[0], 2, 12, 1)
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
