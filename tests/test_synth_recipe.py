"""The seeded synthetic inputs follow the stated workload recipes: sizes,
camera rigs and resolutions, attribute distributions, the batching and
serving draws, and round-to-nearest-even BF16 storage."""
import math

import numpy as np

from paper_2606_09074_gb300 import synth


def camera_centres(cams):
    """Camera centres c = -R^T t of world-to-camera records."""
    R = np.asarray(cams["R"], dtype=np.float64).reshape(-1, 3, 3)
    t = np.asarray(cams["t"], dtype=np.float64)
    return -np.einsum("vji,vj->vi", R, t)


def test_small_scene_recipe():
    w = synth.config0()
    assert w.scene.n == 10_000 and len(w.cams) == 16 and w.ratios == (0.5,)
    assert np.all(w.cams["width"] == 640) and np.all(w.cams["height"] == 480)
    assert np.all(w.cams["fx"] == 512.0) and np.all(w.cams["fy"] == 512.0)
    assert np.all(w.cams["cx"] == 320.0) and np.all(w.cams["cy"] == 240.0)
    assert np.allclose(w.cams["znear"], 0.01) and np.allclose(w.cams["zfar"], 100.0)
    c = camera_centres(w.cams)
    assert np.allclose(np.hypot(c[:, 0], c[:, 1]), 4.0, atol=1e-5) and np.allclose(c[:, 2], 1.0, atol=1e-5)
    # every camera looks at the origin: its optical axis (third row of R) points there
    R = np.asarray(w.cams["R"], dtype=np.float64).reshape(-1, 3, 3)
    to_origin = -c / np.linalg.norm(c, axis=1, keepdims=True)
    assert np.allclose(np.einsum("vi,vi->v", R[:, 2], to_origin), 1.0, atol=1e-5)
    # rotations are orthonormal
    assert np.allclose(np.einsum("vij,vkj->vik", R, R), np.eye(3)[None], atol=1e-5)
    mu = w.scene.pos
    assert np.all(np.abs(mu) <= 6.0)
    assert abs(np.std(mu) - 2.0) < 0.1  # N(0, 2^2), clipped at 3 sigma
    a = w.scene.attr
    assert abs(a[0:3].mean() + 4.5) < 0.05 and abs(a[0:3].std() - 1.0) < 0.05  # log-scales N(-4.5, 1)
    assert np.allclose(np.linalg.norm(a[3:7], axis=0), 1.0, atol=1e-5)  # unit quaternions
    assert abs(a[7].std() - 2.0) < 0.1  # opacity logits N(0, 2)
    assert abs(a[8:11].std() - 0.5) < 0.02 and abs(a[11:56].std() - 0.1) < 0.005  # SH DC, rest


def test_core_shell_recipe():
    w = synth.config_core_shell(seed=5, n=200_000, v=60, width=1297, height=840)
    r = np.linalg.norm(w.scene.pos.astype(np.float64), axis=0)
    shell = (r >= 6.0) & (r <= 10.0)
    # the core N(0, 1.5^2) reaches radius 6 with probability ~1e-3, so the
    # shell fraction is 30% within sampling error
    assert abs(shell.mean() - 0.30) < 0.01
    c = camera_centres(w.cams)
    rc = np.linalg.norm(c, axis=1)
    assert np.all((rc >= 3.5 - 1e-4) & (rc <= 4.5 + 1e-4)) and np.all(c[:, 2] >= -1e-6)
    assert np.all(w.cams["fx"] == 1100.0) and np.all(w.cams["width"] == 1297)
    assert synth.config1(n=1000).ratios == (0.5, 0.66, 0.9)


def test_batch_and_serving_draws():
    res = {tuple(x) for x in synth.RESOLUTIONS}
    for sd in range(100, 164, 21):
        w = synth.batch_scene(sd)
        assert 50_000 <= w.scene.n <= 2_000_000 and 50 <= len(w.cams) <= 300
        assert (int(w.cams["width"][0]), int(w.cams["height"][0])) in res
        assert w.scene.dtype == "bf16" and w.ratios == (0.66,)
    specs = [synth.job_spec(sd) for sd in range(1000, 1400)]
    assert all(50 <= s[1] <= 300 and tuple(s[2]) in res for s in specs)
    assert all(50_000 <= s[0] <= 3_500_000 for s in specs)
    assert {s[3] for s in specs} == {0.5, 0.66, 0.9}
    # N log-uniform: the mean of ln N is the midpoint of the log range
    mid = 0.5 * (math.log(50_000) + math.log(3_500_000))
    assert abs(np.mean([math.log(s[0]) for s in specs]) - mid) < 0.15
    t = synth.job_arrivals(2000, rate=20.0, seed=999)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.05) < 0.005  # exponential gaps, 20 per second


def test_bf16_storage_rounds_to_nearest_even():
    x = np.array([1.0, 1.00390625, 1.01171875, -3.14159, 1e-30, 65504.0, 0.0, -0.0], dtype=np.float32)
    b = synth.f32_to_bf16_bits(x)
    y = synth.bf16_bits_to_f32(b)
    # halfway cases go to the even neighbour: 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    assert y[0] == 1.0 and y[1] == 1.0 and y[2] == np.float32(1.015625)
    assert np.all(np.abs(y[3:6] - x[3:6]) <= np.abs(x[3:6]) * 2.0 ** -8)
    assert np.signbit(y[7]) and y[6] == 0.0
    w = synth.config0(n=500)
    s16 = w.scene.to_bf16()
    assert s16.dtype == "bf16" and np.array_equal(s16.pos, w.scene.pos)  # positions stay float32
    back = synth.bf16_bits_to_f32(s16.attr)
    assert np.all(np.abs(back - w.scene.attr) <= np.abs(w.scene.attr) * 2.0 ** -8)
    # the mixed form: log-scale rows untouched, every other row as bf16 rounds it
    s16s = w.scene.to_bf16s()
    assert s16s.dtype == "bf16s" and s16s.attr.dtype == np.float32
    assert np.array_equal(s16s.attr[:3], w.scene.attr[:3])
    assert np.array_equal(s16s.attr[3:], back[3:])
    assert np.array_equal(s16s.params_f64()[3:], s16s.attr.astype(np.float64))
