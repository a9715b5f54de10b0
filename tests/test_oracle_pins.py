"""Pins of the FP64 oracle against things other than itself: closed forms
derived from the paper's equations, finite differences, textbook rotations,
library eigen-solvers, invariants of the method and brute force on tiny
inputs.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_09074_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C0 = 0.28209479177387814


def cam_from(d):
    c = np.zeros(1, dtype=synth.CAMERA_DTYPE)[0]
    c["R"] = d["R"]; c["t"] = d["t"]
    for k in ("fx", "fy", "cx", "cy", "width", "height", "znear", "zfar"):
        c[k] = d[k]
    return c


def one_primitive(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, dc=(0.3, -0.2, 0.1), rest=0.0):
    g = np.zeros((59, 1))
    g[0:3, 0] = mean
    g[3:6, 0] = log_scale
    g[6:10, 0] = quat
    g[10, 0] = logit
    g[11:14, 0] = dc
    g[14:59, 0] = rest
    return g


def ident_cam(fx=512.0, fy=512.0, w=640, h=480, cx=None, cy=None):
    return cam_from({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": fx, "fy": fy,
                     "cx": w / 2 if cx is None else cx, "cy": h / 2 if cy is None else cy,
                     "width": w, "height": h, "znear": 0.01, "zfar": 100.0})


# ------------------------------------------------------------ golden file

def load_gold():
    with open(os.path.join(GOLD, "single_primitive_closed_forms.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", load_gold()["cases"], ids=lambda c: c["name"])
def test_golden_single_primitive(case):
    cam = cam_from(case["camera"])
    gd = case["gaussian"]
    g = one_primitive(gd["mean"], gd["log_scale"], gd["quat"], gd["logit"])
    oc = oracle.cameras(np.array([cam], dtype=synth.CAMERA_DTYPE))[0]
    tc = oracle.to_camera(oc, g[0:3, 0])
    if "uv" in case:
        np.testing.assert_allclose(oracle.project(oc, tc), case["uv"], rtol=1e-12, atol=1e-9)
    if "J" in case:
        np.testing.assert_allclose(oracle.jacobian(oc, tc), case["J"], rtol=1e-12, atol=1e-12)
    alpha, s, R, Sigma = oracle.activate(g, 0)
    if "alpha" in case:
        assert alpha == pytest.approx(case["alpha"], rel=1e-14)
    if "cov2d" in case:
        np.testing.assert_allclose(oracle.cov2d(oc, tc, Sigma), case["cov2d"], rtol=1e-10, atol=1e-9)
    vis, border = oracle.visible(oc, g[0:3, 0], Sigma)
    assert vis == case["visible"] and not border
    o = oracle.score(g, np.array([cam], dtype=synth.CAMERA_DTYPE))
    assert o["S"][0] == pytest.approx(case["S"], rel=1e-13, abs=0)
    assert o["scores"][0] == pytest.approx(case["score_n1"], rel=1e-12, abs=0)


# --------------------------------------------------------------- Eq. 1

def test_quaternion_rotation_textbook():
    """R(q) for a rotation by theta about z (q = (cos th/2, 0, 0, sin th/2))
    is the textbook planar rotation; a non-unit q gives the same R."""
    th = 0.7
    g = one_primitive((0, 0, 0), (0, 0, 0), (3 * math.cos(th / 2), 0, 0, 3 * math.sin(th / 2)))
    _, _, R, _ = oracle.activate(g, 0)
    ref = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(R, ref, atol=1e-14)
    # about x
    g = one_primitive((0, 0, 0), (0, 0, 0), (math.cos(th / 2), math.sin(th / 2), 0, 0))
    _, _, R, _ = oracle.activate(g, 0)
    ref = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    np.testing.assert_allclose(R, ref, atol=1e-14)


def test_activation_random():
    """R orthonormal with det +1; Sigma symmetric PD with eigenvalues s^2
    (checked with LAPACK); alpha = sigmoid(logit) at textbook points."""
    w = synth.config0(n=200)
    g = w.scene.params_f64()
    for i in range(0, 200, 7):
        alpha, s, R, Sigma = oracle.activate(g, i)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
        np.testing.assert_allclose(Sigma, Sigma.T, atol=1e-15 * np.abs(Sigma).max(), rtol=0)
        ev = np.sort(np.linalg.eigvalsh(Sigma))
        np.testing.assert_allclose(ev, np.sort(np.exp(2 * g[3:6, i])), rtol=1e-9,
                                   atol=1e-14 * ev.max())
        np.testing.assert_allclose(s, np.exp(g[3:6, i]), rtol=1e-15)
        assert 0.0 < alpha < 1.0
    for logit, a in ((0.0, 0.5), (math.log(3.0), 0.75), (-math.log(3.0), 0.25)):
        g = one_primitive((0, 0, 0), (0, 0, 0), logit=logit)
        assert oracle.activate(g, 0)[0] == pytest.approx(a, rel=1e-15)


def test_magnitudes_hand():
    """R1 magnitudes: gem = product of the two largest scales, col = |c|_2
    over the 48 SH coefficients, opa = alpha."""
    g = one_primitive((0, 0, 0), (math.log(0.2), math.log(0.05), math.log(0.3)),
                      logit=math.log(3.0), dc=(1.0, 2.0, 2.0), rest=0.0)
    m = oracle.magnitudes(g, 0)
    assert m[0] == pytest.approx(0.3 * 0.2, rel=1e-14)
    assert m[1] == pytest.approx(3.0, rel=1e-15)
    assert m[2] == pytest.approx(0.75, rel=1e-15)
    g[14:59, 0] = 0.5  # 45 coefficients of 0.5 add 45/4
    m = oracle.magnitudes(g, 0)
    assert m[1] == pytest.approx(math.sqrt(9.0 + 45 / 4), rel=1e-15)


# ------------------------------------------------------------ Eq. 13-16

def test_jacobian_matches_finite_differences():
    """J_Pi (Eq. 14) equals central differences of Pi (Eq. 13)."""
    w = synth.config0()
    oc = oracle.cameras(w.cams)
    rng = np.random.default_rng(5)
    for k in range(20):
        c = oc[k % len(w.cams)]
        tc = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.5, 8)])
        J = oracle.jacobian(c, tc)
        h = 1e-5
        fd = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd[:, j] = (oracle.project(c, tc + e) - oracle.project(c, tc - e)) / (2 * h)
        np.testing.assert_allclose(J, fd, rtol=1e-7, atol=1e-6)


def test_eq16_limit():
    """Eq. 16: on the axis with f_x = f_y = f, Tr(J^T J) = 2 (f/z)^2."""
    c = oracle.cameras(np.array([ident_cam(fx=700.0, fy=700.0)], dtype=synth.CAMERA_DTYPE))[0]
    for z in (0.5, 2.0, 9.0):
        J = oracle.jacobian(c, np.array([0.0, 0.0, z]))
        assert np.trace(J.T @ J) == pytest.approx(2 * (700.0 / z) ** 2, rel=1e-14)


def test_cov2d_is_linearised_projection():
    """Sigma2D is the covariance of the linearised projection: sample
    offsets d ~ N(0, Sigma), push J W d, compare the sample covariance."""
    w = synth.config0(n=50)
    g = w.scene.params_f64()
    oc = oracle.cameras(w.cams)[0]
    rng = np.random.default_rng(3)
    for i in range(5):
        _, _, _, Sigma = oracle.activate(g, i)
        mu = g[0:3, i]
        tc = oracle.to_camera(oc, mu)
        if tc[2] < 0.5:
            continue
        S2 = oracle.cov2d(oc, tc, Sigma)
        J = oracle.jacobian(oc, tc)
        W = np.array(oc.R[:]).reshape(3, 3)
        d = rng.multivariate_normal(np.zeros(3), Sigma, size=200_000)
        emp = np.cov((J @ W @ d.T))
        np.testing.assert_allclose(S2, emp, rtol=0.02, atol=0.02 * np.abs(S2).max())


def test_cov2d_rigid_motion_invariance():
    """Rotating the world and the camera together leaves Sigma2D unchanged."""
    w = synth.config0(n=20)
    g = w.scene.params_f64()
    cam = w.cams[3]
    oc = oracle.cameras(np.array([cam]))[0]
    th = 0.9
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    cam2 = cam.copy()
    Rc = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    oc2 = oracle.cameras(np.array([cam2]))[0]
    oc2.R[:] = list((Rc @ Rz.T).reshape(-1))
    for i in range(10):
        _, _, _, Sigma = oracle.activate(g, i)
        mu = g[0:3, i]
        a = oracle.cov2d(oc, oracle.to_camera(oc, mu), Sigma)
        b = oracle.cov2d(oc2, oracle.to_camera(oc2, Rz @ mu), Rz @ Sigma @ Rz.T)
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11 * np.abs(a).max())


# ---------------------------------------------------------- visibility

def test_visibility_edges_flagged():
    """A box edge exactly on the image border is visible (closed rectangle)
    and flagged as borderline; just beyond it is not visible."""
    c = oracle.cameras(np.array([ident_cam()], dtype=synth.CAMERA_DTYPE))[0]
    sig = 0.1
    Sigma = np.eye(3) * sig * sig
    z = 4.0
    # on the axis, rx = 3 f sig / z exactly when y = 0; choose x so that u + rx = 0
    # u = 320 + 128 x, rx = 38.4 sqrt(1 + x^2/16); solve u + rx = 0 numerically
    lo, hi = -10.0, -2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 320 + 128 * mid + 38.4 * math.sqrt(1 + mid * mid / 16) > 0:
            hi = mid
        else:
            lo = mid
    v, b = oracle.visible(c, np.array([hi, 0.0, z]), Sigma)
    assert b
    v, b = oracle.visible(c, np.array([hi - 1e-3, 0.0, z]), Sigma)
    assert not v and not b
    v, b = oracle.visible(c, np.array([hi + 1e-3, 0.0, z]), Sigma)
    assert v and not b
    # depth planes
    v, b = oracle.visible(c, np.array([0.0, 0.0, 100.0]), Sigma)
    assert not v and b
    v, b = oracle.visible(c, np.array([0.0, 0.0, 99.0]), Sigma)
    assert v and not b


def test_huge_gaussian_off_image_is_visible():
    c = oracle.cameras(np.array([ident_cam()], dtype=synth.CAMERA_DTYPE))[0]
    v, b = oracle.visible(c, np.array([-20.0, 0.0, 4.0]), np.eye(3) * 9.0)
    assert v and not b


# ----------------------------------------------------------- Eq. features

def test_features_closed_forms():
    """Equal alpha -> F_opa = a(1-a); lumas 0.5 +- d -> F_col = d^2;
    isotropic scale s -> F_gem = s / (s + eta); lambda sums to 1."""
    n = 10
    g = np.zeros((59, n))
    g[6] = 1.0
    g[3:6] = math.log(0.02)
    g[10] = math.log(3.0)
    d = 0.07
    lum = np.where(np.arange(n) % 2 == 0, d, -d)
    g[11:14] = lum / C0  # equal r, g, b -> Y = 0.5 + C0 dc (luma weights sum to 1)
    st = oracle.scene_stats(g)
    assert st["F_opa"] == pytest.approx(0.75 * 0.25, rel=1e-14)
    assert st["F_col"] == pytest.approx(d * d, rel=1e-12)
    assert st["F_gem"] == pytest.approx(0.02 / 0.07, rel=1e-14)
    assert sum(st["lambda"]) == pytest.approx(1.0, abs=1e-15)
    lt = [math.log(0.02 / 0.07 + 0.05) / oracle.E_LN_GEM, d * d / oracle.E_COL, 0.1875 / oracle.E_OPA]
    np.testing.assert_allclose(st["lambda_t"], lt, rtol=1e-12)
    np.testing.assert_allclose(st["lambda"], np.array(lt) / sum(lt), rtol=1e-12)
    # equal lumas: F_col = 0, lambda^col = 0
    g[11:14] = 0.3
    st = oracle.scene_stats(g)
    assert st["F_col"] == pytest.approx(0.0, abs=1e-30)
    assert st["lambda"][1] == pytest.approx(0.0, abs=1e-25)


def test_lambda_clamp_and_equal():
    n = 4
    g = np.zeros((59, n))
    g[6] = 1.0
    # very elongated: max/min ratio 1e3 -> F_gem + eta > 1 -> ln > 0 -> lambda~gem < 0 (E < 0)
    g[3] = math.log(1.0); g[4] = math.log(1e-3); g[5] = math.log(1e-3)
    g[11:14] = np.array([0.1, -0.1, 0.2, -0.2]) / C0
    st = oracle.scene_stats(g)
    assert oracle.E_LN_GEM < 0 and st["lambda_t"][0] == 0.0 and st["lambda"][0] == 0.0
    assert sum(st["lambda"]) == pytest.approx(1.0, abs=1e-15)
    st = oracle.scene_stats(g, oracle.params(flags=oracle.NORM_ATTR | oracle.EQUAL_LAMBDA))
    np.testing.assert_allclose(st["lambda"], [1 / 3] * 3, rtol=1e-15)


def test_calibration_constants_reproduce():
    """The stored Eq. 18 constants are what calibrate.py computes now."""
    from oracle import calibrate
    e = calibrate.compute()
    assert e == pytest.approx((oracle.E_LN_GEM, oracle.E_COL, oracle.E_OPA), rel=1e-12)


def test_header_defaults_match_calibration():
    """The library's default constants in include/refine.h are the oracle's."""
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "refine.h")).read()
    import re
    vals = {}
    for name in ("E_LN_GEM", "E_COL", "E_OPA"):
        m = re.search(r"#define REFINE_DEFAULT_%s\s+\(?([-0-9.eE+]+)" % name, hdr)
        assert m, name
        vals[name] = float(m.group(1))
    assert vals["E_LN_GEM"] == pytest.approx(oracle.E_LN_GEM, rel=1e-15)
    assert vals["E_COL"] == pytest.approx(oracle.E_COL, rel=1e-15)
    assert vals["E_OPA"] == pytest.approx(oracle.E_OPA, rel=1e-15)


# ------------------------------------------------------ Eq. 7 and Eq. 20

def test_two_views_mean():
    """Eq. 20 is a mean over |V| views: one visible view at depth z and one
    view that sees nothing gives alpha / (2 (z^2 + eta)) for N = 1."""
    cams = np.array([ident_cam(), ident_cam()], dtype=synth.CAMERA_DTYPE)
    cams[1]["t"] = [0, 0, -1000.0]  # pushes the primitive behind camera 1
    g = one_primitive((0, 0, 3.0), (math.log(0.05),) * 3, logit=0.0)
    o = oracle.score(g, cams)
    assert o["scores"][0] == pytest.approx(0.5 / (2 * (9.0 + 0.05)), rel=1e-13)


def test_coupling_hand_two_primitives():
    """Eq. 7 by hand for N = 2 and one view: D_i = alpha_i S_i sum_k
    lambda^k m_i^k / mean(m^k)."""
    cams = np.array([ident_cam()], dtype=synth.CAMERA_DTYPE)
    g = np.zeros((59, 2))
    g[0:3, 0] = (0, 0, 2.0); g[0:3, 1] = (0.3, 0.1, 5.0)
    g[3:6, 0] = np.log([0.01, 0.02, 0.03]); g[3:6, 1] = np.log([0.05, 0.05, 0.01])
    g[6] = 1.0
    g[10] = (0.5, -1.0)
    g[11:14, 0] = (0.2, 0.1, 0.0); g[11:14, 1] = (-0.3, 0.0, 0.1)
    o = oracle.score(g, cams)
    lam = o["stats"]["lambda"]
    a = 1 / (1 + np.exp(-g[10]))
    mg = np.array([0.02 * 0.03, 0.05 * 0.05])
    mc = np.array([math.sqrt(0.05), math.sqrt(0.1)])
    S = 1 / (np.array([4.0, 25.0]) + 0.05)
    cpl = lam[0] * mg / mg.mean() + lam[1] * mc / mc.mean() + lam[2] * a / a.mean()
    np.testing.assert_allclose(o["scores"], a * S * cpl, rtol=1e-13)


def test_invariances():
    """Permuting primitives permutes scores; permuting or duplicating views
    changes nothing; a primitive outside every frustum scores 0; a rigid
    motion of scene and cameras changes nothing."""
    w = synth.config0(n=400)
    g = w.scene.params_f64()
    base = oracle.score(g, w.cams)["scores"]
    perm = np.random.default_rng(1).permutation(400)
    np.testing.assert_allclose(oracle.score(g[:, perm], w.cams)["scores"], base[perm], rtol=1e-13)
    vp = np.random.default_rng(2).permutation(len(w.cams))
    np.testing.assert_allclose(oracle.score(g, w.cams[vp])["scores"], base, rtol=1e-12, atol=0)
    np.testing.assert_allclose(oracle.score(g, np.concatenate([w.cams, w.cams]))["scores"], base,
                               rtol=1e-12, atol=0)
    # outside every frustum: far above all cameras (cameras look horizontally-ish at origin)
    g2 = g.copy()
    g2[0:3, 0] = (0.0, 0.0, 5000.0)
    o2 = oracle.score(g2, w.cams)
    assert o2["scores"][0] == 0.0 and o2["S"][0] == 0.0
    # rigid motion: rotate about z by th and translate
    th, tr = 0.4, np.array([0.3, -0.2, 0.1])
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    qr = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    g3 = g.copy()
    g3[0:3] = Rz @ g[0:3] + tr[:, None]
    q = g[6:10]
    w0, x0, y0, z0 = qr
    g3[6] = w0 * q[0] - x0 * q[1] - y0 * q[2] - z0 * q[3]
    g3[7] = w0 * q[1] + x0 * q[0] + y0 * q[3] - z0 * q[2]
    g3[8] = w0 * q[2] - x0 * q[3] + y0 * q[0] + z0 * q[1]
    g3[9] = w0 * q[3] + x0 * q[2] - y0 * q[1] + z0 * q[0]
    cams3 = w.cams.copy()
    for k in range(len(cams3)):
        R = np.asarray(w.cams[k]["R"], dtype=np.float64).reshape(3, 3)
        t = np.asarray(w.cams[k]["t"], dtype=np.float64)
        cams3[k]["R"] = (R @ Rz.T).reshape(-1)
        cams3[k]["t"] = t - R @ Rz.T @ tr
    # cameras are stored in float32: compare against the float32-rounded originals' motion
    oc3 = oracle.cameras(cams3)
    for k in range(len(cams3)):
        R = np.asarray(w.cams[k]["R"], dtype=np.float64).reshape(3, 3)
        t = np.asarray(w.cams[k]["t"], dtype=np.float64)
        oc3[k].R[:] = list((R @ Rz.T).reshape(-1))
        oc3[k].t[:] = list(t - R @ Rz.T @ tr)
    o3 = oracle.score(g3, oc3)
    ok = (o3["nborder"] == 0) & (oracle.score(g, w.cams)["nborder"] == 0)
    np.testing.assert_allclose(o3["scores"][ok], base[ok], rtol=1e-9)


def test_ablation_flags():
    """Table 3 modes: w/o V drops alpha from Eq. 20, w/o P counts visible
    views (P = 1)."""
    w = synth.config0(n=300)
    g = w.scene.params_f64()
    full = oracle.score(g, w.cams)
    novis = oracle.score(g, w.cams, oracle.params(flags=oracle.NORM_ATTR | oracle.NO_VIS))
    a = 1 / (1 + np.exp(-g[10]))
    np.testing.assert_allclose(novis["scores"] * a, full["scores"], rtol=1e-12)
    noproj = oracle.score(g, w.cams, oracle.params(flags=oracle.NORM_ATTR | oracle.NO_PROJ))
    assert np.all(noproj["S"] == np.round(noproj["S"]))
    assert np.all(noproj["S"] <= len(w.cams))


# ------------------------------------------------------------- Sec. 3.3

def brute_select(s, beta):
    n = len(s)
    n_keep = n - int(math.floor(beta * n))
    order = sorted(range(n), key=lambda i: (-s[i], i))
    keep = np.zeros(n, dtype=bool)
    keep[order[:n_keep]] = True
    thr = s[order[n_keep - 1]] if n_keep < n and n_keep > 0 else -math.inf
    return keep, thr, n_keep


def unpack(mask, n):
    bits = np.unpackbits(mask.view(np.uint8), bitorder="little")
    return bits[:n].astype(bool)


@pytest.mark.parametrize("kind", ["random", "equal", "zeros", "signed_zero", "ties", "neg", "inf"])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 64])
def test_select_brute_force(kind, n):
    rng = np.random.default_rng(n * 7 + len(kind))
    if kind == "random":
        s = rng.random(n)
    elif kind == "equal":
        s = np.full(n, 0.25)
    elif kind == "zeros":
        s = np.where(rng.random(n) < 0.6, 0.0, rng.random(n))
    elif kind == "signed_zero":
        s = np.where(rng.random(n) < 0.5, -0.0, 0.0)
        s[rng.random(n) < 0.3] = 1.0
    elif kind == "ties":
        s = rng.integers(0, 3, n).astype(float)
    elif kind == "neg":
        s = rng.normal(size=n)
    else:
        s = np.where(rng.random(n) < 0.3, np.inf, rng.random(n))
    for beta in (0.0, 0.1, 0.5, 0.66, 0.9, 0.999):
        mask, thr, nk = oracle.select(s, beta)
        keep, thr_b, nk_b = brute_select(list(s), beta)
        assert nk == nk_b == n - math.floor(beta * n)
        assert np.array_equal(unpack(mask, n), keep)
        assert thr == thr_b or (math.isinf(thr) and math.isinf(thr_b) and thr < 0 and thr_b < 0)
        # bits past n are clear
        if n % 32:
            assert int(mask[-1]) >> (n % 32) == 0


def test_select_empty():
    mask, thr, nk = oracle.select(np.zeros(0), 0.5)
    assert nk == 0 and mask.size == 0 and thr == -math.inf


def test_compact_order_and_roundtrip():
    rng = np.random.default_rng(9)
    n = 77
    rows = rng.normal(size=(59, n)).astype(np.float32)
    s = rng.random(n)
    mask, _, nk = oracle.select(s, 0.4)
    out, idx = oracle.compact(rows, mask)
    keep = unpack(mask, n)
    assert out.shape == (59, nk) and np.array_equal(idx, np.nonzero(keep)[0])
    assert np.array_equal(out, rows[:, keep])
    assert np.all(np.diff(idx) > 0)
    # bf16-sized rows
    rows16 = rng.integers(0, 65535, size=(56, n)).astype(np.uint16)
    out16, idx16 = oracle.compact(rows16, mask)
    assert np.array_equal(out16, rows16[:, keep]) and np.array_equal(idx16, idx)


def test_borderline_alternatives_helper():
    """valid_alternative accepts S_sure + any subset of borderline terms."""
    o = {"nborder": np.array([0, 2]), "S_sure": np.array([1.0, 2.0]),
         "bterms": np.array([[0, 0, 0, 0], [0.5, 0.25, 0, 0]], dtype=float)}
    assert oracle.valid_alternative(np.array([1.0, 2.75]), o, 1e-6).all()
    assert oracle.valid_alternative(np.array([1.0, 2.25]), o, 1e-6).all()
    assert not oracle.valid_alternative(np.array([1.0, 2.1]), o, 1e-6)[1]


# ------------------------------------------------ Eq. 14 Jacobian energy

@pytest.mark.parametrize("mean", [(0.0, 0.0, 3.0), (0.4, -0.25, 2.0), (-1.1, 0.7, 6.5)])
def test_full_jacobian_term_closed_form(mean):
    """With FULL_JACOBIAN the projection term is Eq. 14's energy of J_Pi
    before the Eq. 16 simplification: for N = 1 and one view,
    D = alpha (fx^2/z^2 + fy^2/z^2 + (fx^2 x^2 + fy^2 y^2)/z^4)."""
    cam = ident_cam(fx=700.0, fy=520.0, w=4000, h=4000)
    cams = np.array([cam], dtype=synth.CAMERA_DTYPE)
    g = one_primitive(mean, (math.log(0.01),) * 3, logit=0.7)
    o = oracle.score(g, cams, oracle.params(flags=oracle.NORM_ATTR | oracle.FULL_JACOBIAN))
    x, y, z = mean
    fx, fy = 700.0, 520.0
    P = fx * fx / z ** 2 + fy * fy / z ** 2 + (fx * fx * x * x + fy * fy * y * y) / z ** 4
    alpha = 1 / (1 + math.exp(-0.7))
    assert o["S"][0] == pytest.approx(P, rel=1e-13)
    assert o["scores"][0] == pytest.approx(alpha * P, rel=1e-12)


def test_full_jacobian_term_matches_finite_differences():
    """The energy equals the squared Frobenius norm of a central-difference
    Jacobian of the projection Pi (Eq. 13), an independent derivative."""
    cam = ident_cam(fx=640.0, fy=610.0, w=5000, h=5000, cx=2400.0, cy=2550.0)
    oc = oracle.cameras(np.array([cam], dtype=synth.CAMERA_DTYPE))[0]
    for tc in ([0.3, -0.2, 2.5], [-1.0, 0.8, 4.0]):
        h = 1e-6
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            J[:, k] = (np.asarray(oracle.project(oc, np.add(tc, e))) - np.asarray(oracle.project(oc, np.subtract(tc, e)))) / (2 * h)
        g = one_primitive(tc, (math.log(0.001),) * 3)
        o = oracle.score(g, np.array([cam], dtype=synth.CAMERA_DTYPE),
                         oracle.params(flags=oracle.NORM_ATTR | oracle.FULL_JACOBIAN))
        assert o["S"][0] == pytest.approx(float((J ** 2).sum()), rel=1e-7)


def test_score_subset_equals_full_score_at_its_indices():
    """score_subset(g, idx) scores the primitives idx of the whole scene: the
    same scores, view sums, borderline records and scene statistics as
    score(g) at those indices, for sorted, unsorted and repeated indices
    (its index path is what the sampled GPU parity checks rely on)."""
    w = synth.random_scene(seed=5, n=3000, v=12, means="core_shell")
    g = w.scene.params_f64()
    full = oracle.score(g, w.cams)
    rng = np.random.default_rng(55)
    for idx in (np.sort(rng.choice(3000, 700, replace=False)), rng.permutation(3000)[:500],
                np.array([0, 2999, 17, 17, 1500, 0], dtype=np.int64)):
        sub = oracle.score_subset(g, idx, w.cams)
        for key in ("scores", "S", "S_sure", "nborder", "bterms"):
            assert np.array_equal(sub[key], full[key][idx]), key
        assert sub["stats"] == full["stats"]
    assert (full["scores"] > 0).mean() > 0.5  # the comparison covers visible primitives
