"""Helpers for the GPU tests: run jobs through the C ABI and through the
oracle on the same seeded inputs."""
import concurrent.futures
import os

import numpy as np

from oracle import ref
from paper_1309_3848_gb300 import synth


def oracle_levels(job):
    """The job's block levels, clamped by the oracle's own geometry."""
    W, H = job.image.width, job.image.height
    L = job.levels
    if job.clamp_levels:
        while L > 0 and ref.grid(W, H, job.num_superpixels, L)[0] == ref.EGEOM:
            L -= 1
    return L


def gpu_levels(binding, job):
    W, H = job.image.width, job.image.height
    if job.clamp_levels:
        return min(job.levels, binding.feasible_levels(W, H, job.num_superpixels))
    return job.levels


def params_for(binding, job):
    L = gpu_levels(binding, job)
    return binding.make_params(job.image.width, job.image.height, job.num_superpixels, L, job.bins_per_channel,
                               job.iters_per_level, job.patch, job.gamma, job.color_space, job.means_iters,
                               job.compactness, job.edge_threshold, job.compact_prior)


def make_images(jobs):
    with concurrent.futures.ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda j: synth.make_image(j.image), jobs))


def oracle_run(job, img):
    r = ref.Ref(job.image.width, job.image.height, job.num_superpixels, oracle_levels(job), job.bins_per_channel,
                job.iters_per_level, job.patch, job.gamma, job.color_space, job.means_iters, job.compactness,
                job.edge_threshold, job.compact_prior)
    return r.run(img)


def oracle_many(jobs, imgs):
    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        return list(ex.map(lambda a: oracle_run(*a), zip(jobs, imgs)))


def gpu_run(binding, torch, jobs, imgs, tuning=None):
    ctx = binding.SeedsContext([params_for(binding, j) for j in jobs])
    if tuning:
        ctx.set_tuning(**tuning)
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full((j.image.height, j.image.width), -1, dtype=torch.int32, device="cuda") for j in jobs]
    ctx.run(d, outs)
    torch.cuda.synchronize()
    ctx.check_status()
    return [o.cpu().numpy() for o in outs], ctx


def first_mismatch(a, b):
    diff = np.argwhere(a != b)
    if len(diff) == 0:
        return None
    y, x = diff[0]
    return "%d differing pixels, first at (x=%d, y=%d): gpu %d oracle %d" % (len(diff), x, y, a[y, x], b[y, x])
