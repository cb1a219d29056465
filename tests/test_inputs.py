"""The seeded synthetic inputs follow their stated recipes: sizes, parameter counts, per-pair
blur and noise ranges, mask density, relative noise levels (readings of Sections 5.1, 5.2),
determinism per seed, independence of replicas, and no arithmetic of the method in the
generator module (it imports neither the checker nor the library)."""
import ast
import os

import numpy as np

from paper_2412_08264_gb300 import synth


def test_batch64_recipe_and_determinism():
    wl = synth.batch_64()
    assert len(wl.pairs) == 64 and wl.n_pixels == 6_549_504 and wl.n_params == 416 and wl.recycle_dim == 16
    for p in wl.pairs:
        assert p.height == p.width and p.height in (128, 192, 256, 384, 512)
        assert 1.0 <= p.blur_sigma <= 2.5 and p.blur_radius == 4 and 0.005 <= p.noise_sigma <= 0.03
    again = synth.batch_64()
    assert all(np.array_equal(a, b) for a, b in zip(wl.x_star, again.x_star))
    assert np.array_equal(wl.theta0, again.theta0)
    other = synth.batch_64(replica=1)                 # another rank's batch: same recipe, new draws
    same = [p.height for p in other.pairs] == [p.height for p in wl.pairs] and \
        all(np.array_equal(a, b) for a, b in zip(wl.x_star, other.x_star))
    assert not same


def test_ground_truths_are_piecewise_constant_rectangles():
    rng = np.random.default_rng(0)
    for h, w in [(32, 32), (64, 90), (28, 28)]:
        x = synth.rectangles_image(rng, h, w)
        assert x.min() >= 0.0 and x.max() <= 1.0
        assert len(np.unique(x)) <= 7           # background + six rectangles


def test_filter_initialisation():
    wl = synth.foe_256()
    F = wl.filter_size ** 2 + 1
    for j in range(wl.n_filters):
        assert wl.theta0[j * F] == -3.0
        assert abs(wl.theta0[j * F + 1:(j + 1) * F].sum()) < 1e-12      # zero-mean taps


def test_inpainting_recipe():
    wl = synth.inpaint_batch()
    assert len(wl.pairs) == 1024 and all((p.height, p.width) == (28, 28) for p in wl.pairs)
    assert wl.n_params == 78 and wl.phi == "sq" and wl.recycle_dim == 30
    m = np.concatenate([mm.ravel() for mm in wl.masks])
    assert abs(m.mean() - 0.3) < 0.005                                   # 30 % of the pixels measured
    xs = np.concatenate([x.ravel()[mm.ravel() > 0] for x, mm in zip(wl.x_star, wl.masks)])
    rel = 0.1 / np.sqrt(np.mean(xs ** 2))
    assert 0.25 < rel < 0.35                                             # relative noise level ~0.3


def test_deconvolution_recipe():
    wl = synth.deconv_batch()
    assert len(wl.pairs) == 512 and all((p.height, p.width) == (64, 64) for p in wl.pairs)
    assert all(p.blur_sigma == 3.0 and p.blur_radius == 4 and p.noise_sigma == 0.08 for p in wl.pairs)
    assert wl.n_params == 624 and wl.phi == "log1p"
    taps = synth.dct_filters(24, 5)
    for j in range(24):
        assert wl.theta0[j * 26] == -3.0
        np.testing.assert_array_equal(wl.theta0[j * 26 + 1:(j + 1) * 26], taps[j].ravel())
    rms = np.sqrt(np.mean(np.concatenate([x.ravel() ** 2 for x in wl.x_star])))
    assert 0.18 < 0.08 / rms < 0.3                                       # near the paper's relative 0.2


def test_generator_module_holds_no_method_code():
    src = open(os.path.join(os.path.dirname(synth.__file__), "synth.py")).read()
    mods = set()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0] if node.level == 0 else "." + (node.module or ""))
    assert mods <= {"numpy", "dataclasses", "typing", "__future__"}, mods
