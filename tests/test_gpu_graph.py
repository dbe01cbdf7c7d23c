"""A batch run recorded in a CUDA graph and replayed on new images of the
same shapes gives the oracle's labels, bit for bit."""
import dataclasses

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
def binding(torch):
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1309_3848_gb300 import binding as b
    return b


def test_batch_run_replays_from_a_cuda_graph(torch, binding):
    jobs = synth.random_small_jobs(55, 7, max_side=220) + [synth.plain_481()[0]]
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    d = [torch.empty((j.image.height, j.image.width, 3), dtype=torch.uint8, device="cuda") for j in jobs]
    outs = [torch.full((j.image.height, j.image.width), -1, dtype=torch.int32, device="cuda") for j in jobs]
    first = gc.make_images(jobs)
    for t, im in zip(d, first):
        t.copy_(torch.from_numpy(im))
    graph = ctx.capture(d, outs)
    for shift in (0, 1000, 2000):
        js = [dataclasses.replace(j, image=dataclasses.replace(j.image, seed=j.image.seed + shift)) for j in jobs]
        imgs = gc.make_images(js)
        for t, im in zip(d, imgs):
            t.copy_(torch.from_numpy(im))
        for o in outs:
            o.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        ctx.check_status()
        for i, (o, w) in enumerate(zip(outs, gc.oracle_many(js, imgs))):
            msg = gc.first_mismatch(o.cpu().numpy(), w)
            assert msg is None, "replay with seed shift %d, image %d: %s" % (shift, i, msg)


def test_superpixels_helper(torch, binding):
    jobs = [synth.plain_481()[0], synth.JobSpec(synth.ImageSpec(160, 120, seed=9, cells=10, sigma=8.0), 80, 5, 4, 2,
                                                clamp_levels=True)]
    imgs = gc.make_images(jobs)
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = binding.superpixels(d, [j.num_superpixels for j in jobs], iters_per_level=2)
    torch.cuda.synchronize()
    for o, w in zip(outs, gc.oracle_many(jobs, imgs)):
        assert gc.first_mismatch(o.cpu().numpy(), w) is None
