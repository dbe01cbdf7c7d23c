"""GPU parity of the compactness prior in the histogram pixel phases (Sec.
6.4; reading R19), of the combined prior (3x3 smoothing, compactness and
edge snapping together), and of SPM on its own (Sec. 6.3; reading R20):
state after every op, whole runs, batches mixing them with plain images,
anytime stops, warp tiles and the allocation-free entry point, bit for bit
against the oracle (labels, histograms and sizes are integers: tolerance 0;
the prior's single-precision scores are evaluated in the same order on both
sides, so the decisions match exactly)."""
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


def prior(job, w=64, **kw):
    return dataclasses.replace(job, compact_prior=w, **kw)


def oracle_ref(job):
    return ref.Ref(job.image.width, job.image.height, job.num_superpixels, gc.oracle_levels(job),
                   job.bins_per_channel, job.iters_per_level, job.patch, job.gamma, job.color_space,
                   job.means_iters, job.compactness, job.edge_threshold, job.compact_prior)


SMALL = synth.JobSpec(synth.ImageSpec(97, 61, seed=6, cells=9, sigma=10.0, gradient=True), 30, 8, 3, 2, 3, (2, 1))
STEP_CASES = {
    "481x321_w64": prior(synth.plain_481()[0], 64),
    "97x61_w400_nopatch": prior(SMALL, 400, patch=0),
    "combined_lab_means": prior(SMALL, 32, color_space=1, means_iters=1, compactness=10, edge_threshold=60),
    "spm_alone": dataclasses.replace(SMALL, iters_per_level=0, means_iters=2, compactness=12),
    "spm_alone_L0": synth.JobSpec(synth.ImageSpec(50, 37, seed=7, cells=5, sigma=15.0), 20, 3, 0, 0, 3, (1, 1),
                                  means_iters=2, compactness=5),
}


@pytest.mark.parametrize("tiles", [1, 2], ids=["per-unit", "tiled"])
@pytest.mark.parametrize("name", sorted(STEP_CASES))
def test_state_matches_after_every_op(torch, binding, name, tiles):
    job = STEP_CASES[name]
    W, H = job.image.width, job.image.height
    img = synth.make_image(job.image)
    L = gc.oracle_levels(job)
    r = oracle_ref(job)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    ctx.set_tuning(block_tiles=tiles)
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
            moved += r.run_phase(level, phase)
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
    assert moved > 0


def check(torch, binding, jobs, tuning=None):
    imgs = gc.make_images(jobs)
    got, _ = gc.gpu_run(binding, torch, jobs, imgs, tuning)
    for i, (a, b) in enumerate(zip(got, gc.oracle_many(jobs, imgs))):
        msg = gc.first_mismatch(a, b)
        assert msg is None, "image %d (%dx%d, prior %d, iters %d, means %d): %s" % (
            i, jobs[i].image.width, jobs[i].image.height, jobs[i].compact_prior, jobs[i].iters_per_level,
            jobs[i].means_iters, msg)


def test_prior_changes_the_labels_and_matches_on_1920x1080(torch, binding):
    job = synth.plain_1080()[0]
    imgs = gc.make_images([job])
    plain = gc.oracle_run(job, imgs[0])
    check(torch, binding, [prior(job, 48)])
    assert not np.array_equal(plain, gc.oracle_run(prior(job, 48), imgs[0]))


def test_batch_mixing_priors_spm_and_plain_images(torch, binding):
    jobs = synth.random_small_jobs(93, 24, max_side=200)
    out = []
    for i, j in enumerate(jobs):
        if i % 4 == 0:
            out.append(prior(j, (16, 128, 1024)[i % 3]))
        elif i % 4 == 1:
            out.append(dataclasses.replace(j, iters_per_level=0, means_iters=1 + i % 2, compactness=i % 7))
        elif i % 4 == 2:
            out.append(prior(j, 80, edge_threshold=40, color_space=1))
        else:
            out.append(j)
    for tuning in (None, dict(block_tiles=2, pixel_tile_rows=2), dict(small_block_area=1, hist_layout=1)):
        check(torch, binding, out, tuning)


def test_anytime_stops_with_the_prior(torch, binding):
    job = prior(synth.plain_481()[0], 96)
    img = synth.make_image(job.image)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    d = torch.from_numpy(img).cuda()
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    nops = oracle_ref(job).num_ops()
    for m in list(range(1, nops + 1, 7)) + [nops - 1, nops]:
        ctx.run_anytime([d], [out], max_steps=m)
        steps = ctx.anytime_steps()
        torch.cuda.synchronize()
        ctx.check_status()
        assert steps == m
        msg = gc.first_mismatch(out.cpu().numpy(), oracle_ref(job).run_ops(img, m))
        assert msg is None, "stop after %d steps: %s" % (m, msg)


@pytest.mark.parametrize("job", [prior(synth.plain_481()[0], 200, color_space=1),
                                 dataclasses.replace(synth.plain_481()[0], iters_per_level=0, means_iters=2,
                                                     compactness=9)], ids=["prior_lab", "spm_alone"])
def test_static_entry(torch, binding, job):
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


def test_pixel_phases_from_injected_states_with_the_prior(torch, binding):
    """Ragged states (from the oracle's sequential mode) injected through the
    test hook, which recounts histograms and the prior's coordinate sums:
    each pixel phase from them equals the oracle's."""
    rng = np.random.default_rng(5)
    job = prior(synth.JobSpec(synth.ImageSpec(80, 60, seed=8, cells=10, sigma=14.0), 24, 5, 2, 3), 160)
    W, H = 80, 60
    img = synth.make_image(job.image)
    d = torch.from_numpy(img).cuda()
    r = oracle_ref(job)
    ctx = binding.SeedsContext([gc.params_for(binding, job)])
    ctx.run_ops([d], 0, 1)  # bins
    r.sequential(img, seed=int(rng.integers(0, 1 << 30)))
    state = r.labels()
    ops = [(op,) + ctx.op_info(0, op) for op in range(ctx.num_ops(0))]
    for op, kind, level, phase in [o for o in ops if o[1] == 1 and o[2] == 0][:4]:
        r.set_labels(state)
        ctx.set_labels(0, 0, state)
        ctx.run_ops([d], op, op + 1)
        ctx.check_status()
        assert r.run_phase(0, phase) > 0
        lab, hist, sizes, _ = ctx.read_state(0, 0, (H, W), r.nbins, W * H)
        assert gc.first_mismatch(lab, r.labels()) is None
        h, s = r.hist()
        assert np.array_equal(hist, h) and np.array_equal(sizes, s)
