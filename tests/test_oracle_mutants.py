"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of seeds_ref.c with one planted mistake (a dropped
term, a wrong sign, a transposed operand, a shifted index ...) on the CPU and
runs the pin suite against it in a subprocess; the suite has to fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "seeds_ref.c")

MUTANTS = {
    "G term loses |K_p|": ("(G_n + Kp - G_k)", "(G_n - G_k)"),
    "candidate G difference sign": ("(i128)(G - G_b)", "(i128)(G_b - G)"),
    "block stay test transposed": ("S_n * s_rest > S_stay * st->size[n]", "S_n * st->size[n] > S_stay * s_rest"),
    "intersection scales by the wrong size": ("(i128)Lh[j] * sA", "(i128)Lh[j] * m"),
    "patch window one column short": ("qx <= ix + 1; ++qx)\n                    if (in_image(st, qx, qy) && st->lab",
                                      "qx <= ix; ++qx)\n                    if (in_image(st, qx, qy) && st->lab"),
    "ring test ignores which cells are 4-neighbours": ("if (r & 1) run_has_4 = 1;", "run_has_4 = 1;"),
    "stay histogram keeps the moving pixel": ("(i128)(a_k - 1) * s_n", "(i128)a_k * s_n"),
    "bin order B-major": ("br * B * B + bg * B + bb", "bb * B * B + bg * B + br"),
    "size not decremented on a move": ("            st->size[k] -= 1;\n", "\n"),
    "ties go to the largest label": ("if (!(diff > 0)) continue;", "if (diff < 0) continue;"),
    "LAB line segment loses its offset": ("(24389 * T + ((int64_t)432 << 44))", "(24389 * T)"),
    "LAB a* from the wrong channel pair": ("500 * (f[0] - f[1])", "500 * (f[0] - f[2])"),
    "LAB without the sRGB decoding curve": ("pow((c + 0.055) / 1.055, 2.4)", "c"),
    "LAB bins from the RGB bytes": ("if (st->p.color_space == 1) rgb_to_lab8", "if (0) rgb_to_lab8"),
    "means distance drops the spatial term": ("return dc + st->means_w * ds;", "return dc;"),
    "means ties go to the largest label": ("if (best < 0 || d < db) {", "if (best < 0 || d <= db) {"),
    "means sums the bins, not the colour codes": ("m[0] += st->code[3 * i];", "m[0] += st->bin[i];"),
    "means centroid row from x": ("m[4] += y;", "m[4] += x;"),
    "edge snapping ignores whether the neighbour's label differs": ("if (st->lab[j] != k && code_l1(st, i, j) >= tau)",
                                                                     "if (code_l1(st, i, j) >= tau)"),
    "edge threshold taken as strict": ("code_l1(st, i, j) >= tau) return 1;", "code_l1(st, i, j) > tau) return 1;"),
    "edge snapping skipped in the means phases": ("    if (edge_frozen(st, x, y, k)) return -1;\n    int best = -1;\n    float db",
                                                  "    int best = -1;\n    float db"),
    "anytime prefix skips the descent op": ("        if (level > 0) ++done; /* the descent", "        /* the descent"),
    "anytime prefix runs one phase too many": ("if (done >= nops) return total;", "if (done > nops) return total;"),
    "compact prior with the sign of the distance term flipped": ("return (t1 + t2) - t3;", "return (t1 + t2) + t3;"),
    "compact prior stay centre without the pixel": (
        "st->size[k] - 1, st->size[k], Gk);", "st->size[k] - 1, st->size[k] - 1, Gk);"),
    "compact prior centre row from x": ("float gy = (float)y - (float)m[4] * r;", "float gy = (float)y - (float)m[3] * r;"),
    "compact prior drops the boundary term": ("float t2 = st->gamma_f * (float)G;", "float t2 = 0.0f * (float)G;"),
    "compact prior ignores the superpixel area": (
        "(float)((int64_t)p->compact_prior * 81 * st->K) / (float)((int64_t)16 * N)",
        "(float)((int64_t)p->compact_prior * 81) / (float)16"),
    "compact prior centres taken once, not at every phase start": (
        "    if (level == 0 && st->p.compact_prior > 0) means_recount(st); /* R19: centres at phase start */\n",
        "    if (level == 0 && st->p.compact_prior > 0 && phase == 0 && 0) means_recount(st);\n"),
    "sequential visiting order by Sattolo's shuffle": ("splitmix64(rng) % (uint64_t)(u + 1)", "splitmix64(rng) % (uint64_t)u"),
    "sequential generator loses its second mix": ("z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;", "z = z ^ (z >> 27);"),
    "sequential candidate pick never takes the last candidate": (
        "return (int)(splitmix64(rng) % (uint64_t)nc);", "return (int)(splitmix64(rng) % (uint64_t)(nc > 1 ? nc - 1 : 1));"),
    "SPM alone runs one histogram iteration": (
        "        for (int it = 0; it < st->p.iters_per_level; ++it)\n            for (int phase = 0; phase < 4; ++phase) total += ref_run_phase(st, level, phase);",
        "        for (int it = 0; it < (st->p.iters_per_level ? st->p.iters_per_level : 1); ++it)\n            for (int phase = 0; phase < 4; ++phase) total += ref_run_phase(st, level, phase);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: %s" % name
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    lib = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib), str(c), "-lm"], check=True)
    env = dict(os.environ, SEEDS_REF_LIB=str(lib))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, "pins passed with the mutant '%s'" % name
