"""Quality of the readings against a known truth (Sec. 6.1 metrics on
synthetic Voronoi images, whose cells are the ground-truth segments): the
parallel parity schedule (readings R5, R6) improves the grid as much as the
paper's sequential order does (the oracle's sequential mode, R14)."""
import pytest

from oracle import ref
from paper_1309_3848_gb300 import metrics as quality
from paper_1309_3848_gb300 import synth


@pytest.mark.parametrize("seed", range(3))
def test_parallel_schedule_matches_the_sequential_order(seed):
    spec = synth.ImageSpec(200, 150, seed=70 + seed, cells=14, sigma=8.0, gradient=True)
    img, truth = synth.make_image(spec), synth.voronoi_truth(spec)
    args = (spec.width, spec.height, 80, 3, 5, 2)
    grid = ref.Ref(*args).run_ops(img, 1)
    par = ref.Ref(*args).run(img)
    seq, _, _ = ref.Ref(*args).sequential(img, seed=seed)
    g, p, s = [(quality.cue(x, truth), quality.br(x, truth), quality.asa(x, truth)) for x in (grid, par, seq)]
    # both schedules move the grid's boundaries onto the true edges
    assert p[0] < g[0] / 10 and s[0] < g[0] / 10
    assert p[1] > g[1] + 0.4 and s[1] > g[1] + 0.4
    assert p[2] > 0.99
    # and the parallel one does about as well as the sequential one
    assert p[0] <= 1.5 * s[0] + 0.002
    assert p[1] >= s[1] - 0.02


def test_metrics_on_known_cases():
    import numpy as np
    truth = np.zeros((4, 6), np.int32)
    truth[:, 3:] = 1
    assert quality.cue(truth, truth) == 0 and quality.asa(truth, truth) == 1 and quality.br(truth, truth) == 1
    lab = truth.copy()
    lab[0, 3] = 0  # one pixel of segment 1 given to superpixel 0
    assert quality.cue(lab, truth) == pytest.approx(1 / 24)
    assert quality.asa(lab, truth) == pytest.approx(23 / 24)
    # UE counts superpixel 0 (13 px, 1 outside g0) at g0, and both superpixels at g1: 1 + 12 + 0
    assert quality.ue(lab, truth) == pytest.approx(13 / 24)
    grid = np.zeros((4, 6), np.int32)  # one superpixel: no boundary recalled
    assert quality.br(grid, truth) == 0
