"""GPU parity of anytime termination (Sec. 5.4): a launch stopped after n
steps, by a step limit or by a device-time budget, leaves every image with
the oracle's partition after its first n ops, bit for bit."""
import concurrent.futures
import os

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


def oracle_ref(job):
    return ref.Ref(job.image.width, job.image.height, job.num_superpixels, gc.oracle_levels(job),
                   job.bins_per_channel, job.iters_per_level, job.patch, job.gamma, job.color_space,
                   job.means_iters, job.compactness, job.edge_threshold)


def oracle_prefixes(job, img, counts):
    """{n: oracle labels after the first n ops} for the given op counts."""
    def one(n):
        return n, oracle_ref(job).run_ops(img, n)
    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        return dict(ex.map(one, sorted(set(counts))))


def setup(torch, binding, jobs):
    imgs = gc.make_images(jobs)
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full((j.image.height, j.image.width), -1, dtype=torch.int32, device="cuda") for j in jobs]
    return imgs, ctx, d, outs


def run(torch, ctx, d, outs, max_steps=0, budget_ns=0):
    for o in outs:
        o.fill_(-1)
    ctx.run_anytime(d, outs, max_steps=max_steps, budget_ns=budget_ns)
    steps = ctx.anytime_steps()
    torch.cuda.synchronize()
    ctx.check_status()
    return steps, [o.cpu().numpy() for o in outs]


def test_every_stop_point_of_one_image(torch, binding):
    job = synth.plain_481()[0]
    imgs, ctx, d, outs = setup(torch, binding, [job])
    nops = oracle_ref(job).num_ops()
    want = oracle_prefixes(job, imgs[0], range(1, nops + 1))
    for m in range(1, nops + 3):
        steps, got = run(torch, ctx, d, outs, max_steps=m)
        assert steps == min(m, nops)
        msg = gc.first_mismatch(got[0], want[steps])
        assert msg is None, "stop after %d steps: %s" % (steps, msg)


MIXED = [
    synth.JobSpec(synth.ImageSpec(481, 321, seed=31, cells=12, sigma=8.0, gradient=True), 200, 5, 4, 2),
    synth.JobSpec(synth.ImageSpec(320, 240, seed=32, cells=30, sigma=8.0), 900, 5, 4, 2, clamp_levels=True),
    synth.JobSpec(synth.ImageSpec(97, 61, seed=33, cells=9, sigma=10.0), 30, 8, 3, 3, 3, (2, 1)),
    synth.JobSpec(synth.ImageSpec(50, 37, seed=34, cells=5, sigma=15.0), 20, 3, 0, 3, 0, (1, 1)),
    synth.JobSpec(synth.ImageSpec(640, 480, seed=35, cells=150, sigma=8.0, texture=True), 600, 5, 4, 2),
]


def test_mixed_batch_stops_every_image_at_the_same_step(torch, binding):
    jobs = MIXED
    imgs, ctx, d, outs = setup(torch, binding, jobs)
    nops = [oracle_ref(j).num_ops() for j in jobs]
    stops = sorted({1, 2, 5, 9, 10, 11, 17, 23, min(nops), min(nops) + 1, max(nops) - 1, max(nops), max(nops) + 4})
    want = [oracle_prefixes(j, im, [min(m, n) for m in stops]) for j, im, n in zip(jobs, imgs, nops)]
    for m in stops:
        steps, got = run(torch, ctx, d, outs, max_steps=m)
        assert steps == min(m, max(nops))
        for i in range(len(jobs)):
            msg = gc.first_mismatch(got[i], want[i][min(m, nops[i])])
            assert msg is None, "stop after %d steps, image %d: %s" % (m, i, msg)


@pytest.mark.parametrize("budget_ns", [1, 30_000, 150_000, 600_000, 10 ** 12])
def test_time_budget_stops_at_a_step_boundary(torch, binding, budget_ns):
    jobs = [synth.plain_1080()[0]]
    imgs, ctx, d, outs = setup(torch, binding, jobs)
    nops = oracle_ref(jobs[0]).num_ops()
    steps, got = run(torch, ctx, d, outs, budget_ns=budget_ns)
    assert 1 <= steps <= nops
    if budget_ns == 1:
        assert steps == 1  # the budget is gone after the first step: the grid
    if budget_ns == 10 ** 12:
        assert steps == nops
    want = oracle_ref(jobs[0]).run_ops(imgs[0], steps)
    msg = gc.first_mismatch(got[0], want)
    assert msg is None, "budget %d ns stopped after %d steps: %s" % (budget_ns, steps, msg)


def test_no_limit_is_the_full_run_and_labels_need_a_new_run(torch, binding):
    jobs = MIXED[:3]
    imgs, ctx, d, outs = setup(torch, binding, jobs)
    steps, got = run(torch, ctx, d, outs)
    assert steps == max(oracle_ref(j).num_ops() for j in jobs)
    for a, b in zip(got, gc.oracle_many(jobs, imgs)):
        assert gc.first_mismatch(a, b) is None
    # after an anytime launch the context holds the stopped state
    with pytest.raises(binding.SeedsError) as e:
        ctx.labels(outs)
    assert e.value.code == binding.SEEDS_ERR_INVALID
    with pytest.raises(binding.SeedsError):
        ctx.run_anytime(d, outs, max_steps=-1)
    # a normal iterate makes the labels available again
    ctx.iterate(d)
    ctx.labels(outs)
    torch.cuda.synchronize()
    ctx.check_status()
    for o, b in zip(outs, gc.oracle_many(jobs, imgs)):
        assert gc.first_mismatch(o.cpu().numpy(), b) is None
