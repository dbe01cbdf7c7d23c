"""Run a set of jobs through the library named by SEEDS_LIB (the
bounds-checked debug build) and compare with the oracle; prints one JSON
line.  Started by test_gpu_debug_bounds.py in a process of its own."""
import ctypes
import dataclasses
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch  # noqa: E402

import gpu_cases as gc  # noqa: E402
from paper_1309_3848_gb300 import binding, synth  # noqa: E402


def main():
    assert binding.LIB_PATH == os.environ["SEEDS_LIB"]
    jobs = synth.plain_481() + synth.random_small_jobs(404, 20, max_side=160)
    jobs += [dataclasses.replace(synth.plain_481()[0], color_space=1, means_iters=2, compactness=9)]
    jobs += [synth.JobSpec(synth.ImageSpec(W, H, seed=W * 7 + H, cells=3, sigma=20.0), K, B, L, 2)
             for W, H, K, B, L in [(1, 1, 1, 5, 0), (1, 40, 3, 4, 0), (40, 1, 3, 4, 0), (2, 2, 1, 16, 0),
                                   (64, 64, 4, 16, 2)]]
    imgs = gc.make_images(jobs)
    results = {}
    for tuning in (None, dict(small_block_area=1, pixel_tile_rows=2), dict(threads_per_block=256, hist_layout=1),
                   dict(block_tiles=2, small_block_area=4), dict(block_tiles=2, pixel_tile_rows=2, hist_layout=1)):
        got, ctx = gc.gpu_run(binding, torch, jobs, imgs, tuning)
        results[str(tuning)] = [gc.first_mismatch(a, b) for a, b in zip(got, gc.oracle_many(jobs, imgs))]
    # an anytime stop inside the block levels
    ctx = binding.SeedsContext([gc.params_for(binding, j) for j in jobs])
    d = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty((j.image.height, j.image.width), dtype=torch.int32, device="cuda") for j in jobs]
    ctx.run_anytime(d, outs, max_steps=7)
    torch.cuda.synchronize()
    ctx.check_status()
    # the allocation-free entry point on the same build: a plain job, a LAB
    # job with means iterations and an edge-snapped one
    static_jobs = [jobs[0], jobs[1 + 20], dataclasses.replace(jobs[2], edge_threshold=30)]
    static = []
    for job in static_jobs:
        img = synth.make_image(job.image)
        p = gc.params_for(binding, job)
        d_img = torch.from_numpy(img).cuda()
        out = torch.full((job.image.height, job.image.width), -1, dtype=torch.int32, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = binding.lib.seeds_run_static(ctypes.byref(p), d_img.data_ptr(), d_img.stride(0), out.data_ptr(),
                                          st.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        want = gc.oracle_run(job, img)
        static.append(None if rc == 0 and int(st.item()) == 0 and gc.first_mismatch(out.cpu().numpy(), want) is None
                      else "rc %d status %d: %s" % (rc, int(st.item()), gc.first_mismatch(out.cpu().numpy(), want)))
    results["static entry"] = static
    print(json.dumps({"mismatches": {k: [m for m in v if m] for k, v in results.items()}, "images": len(jobs)}))


if __name__ == "__main__":
    main()
