"""C ABI checks that need no GPU: the library loads, exports every entry
point that include/seeds.h declares, and its host-side parameter logic
(validation, grid geometry, feasible levels, int64 bound) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "seeds.h")


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1309_3848_gb300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\bint\s+(seeds_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["seeds_create", "seeds_iterate", "seeds_labels", "seeds_num_superpixels", "seeds_destroy",
              "seeds_batch_create", "seeds_batch_iterate", "seeds_debug_set_labels", "seeds_debug_run_ops"]:
        assert n in names


def test_library_exports_every_declared_symbol(binding):
    lib = ctypes.CDLL(binding.LIB_PATH)
    names = declared_functions()
    assert sorted(binding.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_geometry_agrees_with_the_oracle(binding):
    from oracle import ref
    rng = np.random.default_rng(0)
    cases = [(481, 321, 200, 4), (1920, 1080, 1000, 4), (3840, 2160, 5000, 5), (320, 240, 1500, 2),
             (320, 240, 1500, 3), (7, 5, 35, 0), (1, 1, 1, 0)]
    for _ in range(300):
        W, H = int(rng.integers(1, 400)), int(rng.integers(1, 400))
        cases.append((W, H, int(rng.integers(1, max(2, W * H // 3))), int(rng.integers(0, 6))))
    for W, H, K, L in cases:
        p = binding.make_params(W, H, K, L, 5, 1)
        rc, gx, gy = binding.check_params(p)
        rrc, rgx, rgy = ref.grid(W, H, K, L)
        if rrc == ref.EINVAL:
            assert rc == binding.SEEDS_ERR_INVALID
            continue
        assert (gx, gy) == (rgx, rgy), (W, H, K, L)
        assert (rc == binding.SEEDS_ERR_GEOMETRY) == (rrc == ref.EGEOM), (W, H, K, L)
        if rc == 0:
            Lmax = binding.feasible_levels(W, H, K)
            assert Lmax >= L
            assert ref.grid(W, H, K, Lmax)[0] == 0
            assert ref.grid(W, H, K, Lmax + 1)[0] == ref.EGEOM or Lmax + 1 > 12


def test_invalid_parameters(binding):
    bad = [binding.make_params(0, 10, 4, 0, 5, 1), binding.make_params(10, 10, 0, 0, 5, 1),
           binding.make_params(10, 10, 4, 0, 17, 1), binding.make_params(10, 10, 4, 0, 5, 0),
           binding.make_params(10, 10, 4, 0, 5, 1, patch=2), binding.make_params(10, 10, 4, 0, 5, 1, gamma=(1, 0)),
           binding.make_params(10, 10, 4, 13, 5, 1), binding.make_params(10, 10, 4, 0, 5, 1, color_space=2),
           binding.make_params(10, 10, 4, 0, 5, 1, color_space=-1), binding.make_params(10, 10, 4, 0, 5, 1, means_iters=-1),
           binding.make_params(10, 10, 4, 0, 5, 1, means_iters=1001),
           binding.make_params(10, 10, 4, 0, 5, 1, means_iters=1, compactness=1025),
           binding.make_params(10, 10, 4, 0, 5, 1, edge_threshold=-1),
           binding.make_params(10, 10, 4, 0, 5, 1, edge_threshold=766),
           binding.make_params(10, 10, 4, 0, 5, 0), binding.make_params(10, 10, 4, 0, 5, 1, compact_prior=-1),
           binding.make_params(10, 10, 4, 0, 5, 1, compact_prior=1025)]
    for p in bad:
        assert binding.check_params(p)[0] == binding.SEEDS_ERR_INVALID
    assert binding.check_params(binding.make_params(16, 16, 4, 4, 5, 1))[0] == binding.SEEDS_ERR_GEOMETRY
    # exact int64 compares: gamma 1024/1024 on an 8192x8192 image overflows
    assert binding.check_params(binding.make_params(8192, 8192, 1000, 0, 5, 1, gamma=(1024, 1024)))[0] == \
        binding.SEEDS_ERR_INT64


def test_defaults_follow_the_paper(binding):
    p = binding.make_params(1, 1, 1, 0, 1, 1, 0, (0, 1), 1, 7, 9, 11, 13)  # every optional field set
    assert binding.lib.seeds_params_default(ctypes.byref(p), 481, 321, 200) == 0
    assert (p.color_space, p.means_iters, p.compactness, p.edge_threshold, p.compact_prior) == (0, 0, 0, 0, 0)
    # SPM on its own: no histogram iteration, only with means iterations
    assert binding.check_params(binding.make_params(40, 30, 10, 2, 4, 0, means_iters=1))[0] == 0
    p = binding.seeds_params()
    assert binding.lib.seeds_params_default(ctypes.byref(p), 481, 321, 200) == 0
    assert (p.bins_per_channel, p.patch, p.gamma_num, p.gamma_den) == (5, 3, 1, 1)
    assert p.block_levels == 4
    assert binding.lib.seeds_params_default(ctypes.byref(p), 320, 240, 1500) == 0
    assert p.block_levels == 2


def test_footprint_grows_with_the_images(binding):
    a = binding.footprint([binding.make_params(640, 480, 500, 3, 5, 2)])
    b = binding.footprint([binding.make_params(640, 480, 500, 3, 5, 2)] * 3)
    c = binding.footprint([binding.make_params(3840, 2160, 5000, 5, 8, 4)])
    assert a > 640 * 480 * 5 and b >= 3 * a and c > 8 * a


def test_autotune_cache_round_trip(binding, tmp_path):
    p = [binding.make_params(640, 480, 500, 3, 5, 2), binding.make_params(320, 240, 200, 2, 5, 2)]
    k1 = binding.tuning_cache_key(p, "GPU A")
    assert k1 == binding.tuning_cache_key(list(p), "GPU A")
    assert k1 != binding.tuning_cache_key(p[::-1], "GPU A")
    assert k1 != binding.tuning_cache_key(p, "GPU B")
    assert k1 != binding.tuning_cache_key([p[0], binding.make_params(320, 240, 200, 2, 5, 3)], "GPU A")
    path = str(tmp_path / "tune.json")
    assert binding.load_cached_tuning(path, k1) is None
    binding.store_tuning(path, k1, binding.seeds_tuning(512, 1, 1, 9, 2), "two images")
    binding.store_tuning(path, "other", binding.seeds_tuning(1024, 0, 0, 16, 4))
    t = binding.load_cached_tuning(path, k1)
    assert (t.threads_per_block, t.blocks_per_sm, t.hist_layout, t.small_block_area, t.pixel_tile_rows) == \
        (512, 1, 1, 9, 2)
    assert binding.load_cached_tuning(path, "missing") is None


def declaration_comments():
    """Each declared function with the comment text between the previous
    declaration (or section rule) and its own."""
    text = open(HEADER).read()
    out = {}
    prev_end = 0
    for m in re.finditer(r"\bint\s+(seeds_\w+)\s*\(", text):
        chunk = text[prev_end:m.start()]
        comments = " ".join(re.findall(r"/\*.*?\*/", chunk, flags=re.S))
        out[m.group(1)] = comments
        prev_end = text.index(";", m.end()) + 1
    return out


def test_every_declaration_cites_the_paper_or_says_it_has_no_counterpart():
    for name, comment in declaration_comments().items():
        flat = " ".join(re.sub(r"\n\s*\*(?!/)", " ", comment).split())
        assert re.search(r"\b(Sec\.|Prop\.|Eq\.)", flat) or "no counterpart" in flat.lower(), name


def test_entry_points_refuse_a_null_context_or_server(binding):
    """Every call on a context or a server checks its handle before anything
    else: a null one returns SEEDS_ERR_INVALID (no device is touched)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    sigs = re.findall(r"\bint\s+(seeds_\w+)\s*\(\s*(?:const\s+)?(seeds_ctx|seeds_server)\s*\*", text)
    assert len(sigs) >= 30
    for name, _ in sigs:
        fn = getattr(binding.lib, name)
        args = [None if t is ctypes.c_void_p or hasattr(t, "contents") or t is None else t(1)
                for t in fn.argtypes]
        args[0] = None
        assert fn(*args) == binding.SEEDS_ERR_INVALID, name
