"""SEEDS superpixels (arXiv 1309.3848) on GB300: hand-written sm_103a CUDA
behind a C ABI (include/seeds.h), with a thin ctypes binding.

`paper_1309_3848_gb300.binding` loads the compiled library; importing the
package itself loads nothing, so the input generator (`synth`) is usable
without a GPU.
"""
