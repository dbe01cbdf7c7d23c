"""seeds_run_static: the entry point for callers that may not allocate
device memory (a framework that owns the whole device memory through its own
pool, or a latency-critical loop that cannot take cudaMalloc's implicit
synchronisation).  It keeps all of its device state in one static array
inside the library.  Here it is called through the C ABI twice in a row, on
two different images, and each result is checked against the allocating
entry point (seeds_batch_run) on the same input: labels are integers, so the
tolerance is zero.  Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

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


def job_params(binding, job):
    return binding.make_params(job.image.width, job.image.height, job.num_superpixels, job.levels,
                               job.bins_per_channel, job.iters_per_level, job.patch, job.gamma)


def with_allocation(binding, torch, job, d_img):
    ctx = binding.SeedsContext([job_params(binding, job)])
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    ctx.run([d_img], [out])
    torch.cuda.synchronize()
    ctx.check_status()
    return out.cpu().numpy()


def without_allocation(binding, torch, job, d_img):
    p = job_params(binding, job)
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = binding.lib.seeds_run_static(ctypes.byref(p), d_img.data_ptr(), d_img.stride(0), out.data_ptr(),
                                      status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == binding.SEEDS_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out.cpu().numpy()


def test_static_scratch_entry_matches_the_allocating_one(torch, binding):
    jobs = [synth.plain_481()[0],
            synth.JobSpec(synth.ImageSpec(640, 480, seed=41, cells=150, sigma=8.0), 900, 8, 3, 2, 3, (2, 1))]
    for job in jobs:  # two calls in a row; the second reuses the array the first left behind
        d_img = torch.from_numpy(synth.make_image(job.image)).cuda()
        want = with_allocation(binding, torch, job, d_img)
        got = without_allocation(binding, torch, job, d_img)
        assert np.array_equal(got, want), "%d labels differ" % int((got != want).sum())


def test_static_scratch_entry_allocates_nothing(torch, binding):
    """After a first call of the same shape (which loads the kernels), a
    call changes neither the device's free memory nor the caching
    allocator's counters."""
    job = synth.JobSpec(synth.ImageSpec(320, 240, seed=43, cells=40, sigma=8.0), 300, 5, 3, 2)
    d_img = torch.from_numpy(synth.make_image(job.image)).cuda()
    first = without_allocation(binding, torch, job, d_img)
    p = job_params(binding, job)
    out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    rc = binding.lib.seeds_run_static(ctypes.byref(p), d_img.data_ptr(), d_img.stride(0), out.data_ptr(),
                                      status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    stats2 = torch.cuda.memory_stats()
    assert rc == binding.SEEDS_OK and int(status.item()) == 0
    assert free2 == free1, "device free memory moved by %d bytes" % (free1 - free2)
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats2.get(key, 0) == stats1.get(key, 0), key
    assert np.array_equal(out.cpu().numpy(), first)


def test_static_scratch_entry_refuses_images_that_do_not_fit(torch, binding):
    p = binding.make_params(3840, 2160, 5000, 5, 8, 4)
    img = torch.zeros((2160, 3840, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2160, 3840), dtype=torch.int32, device="cuda")
    rc = binding.lib.seeds_run_static(ctypes.byref(p), img.data_ptr(), img.stride(0), out.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == binding.SEEDS_ERR_STATIC_SIZE
