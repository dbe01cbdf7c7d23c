"""GPU parity of the LAB colour space (Sec. 6.2, reading R16): the colour
bins of every sRGB byte triple, and whole runs, bit for bit against the
oracle."""
import ctypes

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


def every_colour():
    """4096 x 4096 image holding each of the 2^24 byte triples once."""
    i = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(i >> 16) & 255, (i >> 8) & 255, i & 255], axis=-1).astype(np.uint8)
    return rgb.reshape(4096, 4096, 3)


@pytest.mark.parametrize("B", [16, 15, 7])
def test_bins_of_every_colour(torch, binding, B):
    img = every_colour()
    W = H = 4096
    p = binding.make_params(W, H, 64, 0, B, 1, 3, (1, 1), 1)
    ctx = binding.SeedsContext([p])
    ctx.run_ops([torch.from_numpy(img).cuda()], 0, 1)  # the initialisation alone
    torch.cuda.synchronize()
    ctx.check_status()
    _, _, _, bins = ctx.read_state(0, 0, (H, W), B ** 3, W * H)
    r = ref.Ref(W, H, 64, 0, B, 1, color_space=1)
    r.init(img)
    want = r.bins().ravel()
    bad = np.nonzero(bins != want)[0]
    assert len(bad) == 0, "%d colours differ, first rgb %s: gpu bin %d oracle bin %d" % (
        len(bad), img.reshape(-1, 3)[bad[0]].tolist(), bins[bad[0]], want[bad[0]])


def lab(job):
    return synth.JobSpec(job.image, job.num_superpixels, job.bins_per_channel, job.levels, job.iters_per_level,
                         job.patch, job.gamma, job.clamp_levels, color_space=1)


def check(torch, binding, jobs):
    imgs = gc.make_images(jobs)
    got, _ = gc.gpu_run(binding, torch, jobs, imgs)
    for i, (a, b) in enumerate(zip(got, gc.oracle_many(jobs, imgs))):
        msg = gc.first_mismatch(a, b)
        assert msg is None, "image %d (%dx%d, colour space %d): %s" % (
            i, jobs[i].image.width, jobs[i].image.height, jobs[i].color_space, msg)


def test_plain_481x321_in_lab(torch, binding):
    check(torch, binding, [lab(synth.plain_481()[0])])


def test_plain_1920x1080_in_lab(torch, binding):
    check(torch, binding, [lab(synth.plain_1080()[0])])


def test_batch_mixing_colour_spaces(torch, binding):
    jobs = synth.random_small_jobs(77, 24, max_side=200)
    jobs = [lab(j) if i % 2 == 0 else j for i, j in enumerate(jobs)]
    jobs.append(lab(synth.JobSpec(synth.ImageSpec(3840, 2160, seed=78, cells=1000, sigma=5.0), 5000, 8, 5, 2)))
    check(torch, binding, jobs)


def test_static_entry_in_lab(torch, binding):
    job = lab(synth.plain_481()[0])
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

