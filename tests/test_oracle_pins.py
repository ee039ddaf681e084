"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Library routines (scipy's spherical harmonics and rotations), sigma-point projection of
the exact pinhole model, closed forms for one and two splats, the invariants the paper
states (hierarchical == flat, Eq. 5 == Eq. 2; crisp partial images when the optical axis
lies on a dividing plane), brute force on tiny inputs, and finite differences.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sps
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2406_11836_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers
class _S:
    """Minimal scene holder (float64 arrays allowed for finite differences)."""

    def __init__(self, means, log_scales, quats, logits, sh, deg):
        self.means, self.log_scales, self.quats = means, log_scales, quats
        self.opacity_logits, self.sh, self.sh_degree = logits, sh, deg

    def copy(self):
        return _S(*(np.array(a, np.float64, copy=True) for a in
                    (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)), self.sh_degree)


def rand_scene(n, seed, extent=1.0, log_scale=(-2.5, 0.4), deg=0):
    r = np.random.default_rng(seed)
    q = r.normal(size=(n, 4))
    nsh = (deg + 1) ** 2
    sh = r.uniform(0, 1, (n, nsh, 3)) if deg == 0 else r.normal(0, 0.3, (n, nsh, 3))
    return _S(r.uniform(-extent, extent, (n, 3)).astype(np.float32),
              r.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32),
              (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32),
              r.normal(0, 1, n).astype(np.float32), sh.astype(np.float32), deg)


def real_sh_scipy(l, m, d):
    """Real SH with Condon-Shortley phase from scipy's complex Y_l^m."""
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    y = sps.sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2) * y.real
    if m < 0:
        return math.sqrt(2) * y.imag
    return y.real


def unit_dirs(n, seed):
    r = np.random.default_rng(seed)
    d = r.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def exact_projection(cam, x):
    V = np.asarray(cam.viewmat, np.float32).astype(np.float64)
    p = x @ V[:3, :3].T + V[:3, 3]
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    return np.stack([fx * p[:, 0] / p[:, 2] + cx, fy * p[:, 1] / p[:, 2] + cy], axis=1), p


# --------------------------------------------------------------------------- SH basis
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_sh_basis_matches_scipy(deg):
    d = unit_dirs(200, deg)
    Y, _ = O.sh_basis(deg, d)
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, l * l + m + l], real_sh_scipy(l, m, d), atol=1e-13)


def test_sh_gradient_tangential_matches_fd():
    d = unit_dirs(50, 3)
    Y, dY = O.sh_basis(3, d)
    r = np.random.default_rng(9)
    for i in range(d.shape[0]):
        tau = np.cross(d[i], r.normal(size=3))
        tau /= np.linalg.norm(tau)
        h = 1e-6
        dp = (d[i] + h * tau) / np.linalg.norm(d[i] + h * tau)
        dm = (d[i] - h * tau) / np.linalg.norm(d[i] - h * tau)
        fd = (O.sh_basis(3, dp[None])[0][0] - O.sh_basis(3, dm[None])[0][0]) / (2 * h)
        np.testing.assert_allclose(dY[i] @ tau, fd, atol=1e-8)


# --------------------------------------------------------------------------- projection (Sec. 3.1)
def test_ewa_covariance_matches_sigma_points():
    """Sigma' - dilation*I equals the covariance of the exactly projected sigma points of a
    tiny Gaussian (the linearisation is exact in the limit); rotation from scipy."""
    r = np.random.default_rng(3)
    cam = W.look_at((2.0, -3.0, 1.5), (0.1, 0.2, -0.1), 96, 64, up=(0, 0, 1))
    for trial in range(20):
        mu = r.uniform(-0.6, 0.6, 3)
        q = r.normal(size=4)
        q /= np.linalg.norm(q)
        s = np.exp(r.normal(-9.5, 0.5, 3))
        sc = _S(mu[None].astype(np.float32), np.log(s)[None].astype(np.float32), q[None].astype(np.float32),
                np.zeros(1, np.float32), np.zeros((1, 1, 3), np.float32), 0)
        mu64 = sc.means[0].astype(np.float64)
        s64 = np.exp(sc.log_scales[0].astype(np.float64))
        q64 = sc.quats[0].astype(np.float64)
        Rq = Rotation.from_quat([q64[1], q64[2], q64[3], q64[0]]).as_matrix()
        Lm = Rq @ np.diag(s64)
        pts = np.concatenate([mu64 + math.sqrt(3) * Lm[:, j] * sgn for j in range(3) for sgn in (1, -1)]).reshape(6, 3)
        xy, _ = exact_projection(cam, pts)
        c = xy - xy.mean(0)
        cov = c.T @ c / 6.0
        pr = O.project(sc, cam)
        dil = float(np.float32(0.3))      # the dilation reaches the renderer as float32
        got = np.array([[pr["cov_xx"][0] - dil, pr["cov_xy"][0]], [pr["cov_xy"][0], pr["cov_yy"][0] - dil]])
        np.testing.assert_allclose(got, cov, rtol=1e-5, atol=1e-12 * np.abs(cov).max())
        mean, p = exact_projection(cam, mu64[None])
        np.testing.assert_allclose([pr["mean_x"][0], pr["mean_y"][0]], mean[0], rtol=1e-13)
        assert abs(pr["z"][0] - p[0, 2]) < 1e-12
        C = np.array([[pr["conic_a"][0], pr["conic_b"][0]], [pr["conic_b"][0], pr["conic_c"][0]]])
        S = np.array([[pr["cov_xx"][0], pr["cov_xy"][0]], [pr["cov_xy"][0], pr["cov_yy"][0]]])
        np.testing.assert_allclose(C @ S, np.eye(2), atol=1e-10)


def test_isotropic_on_axis_closed_form():
    """Isotropic splat of scale s on the optical axis at depth z: Sigma' = ((f s/z)^2 + 0.3) I,
    independent of the quaternion."""
    cam = W.axis_camera((0.0, 0.0, -3.0), 128, 128)
    f = float(np.float32(cam.fx))
    for q in np.random.default_rng(1).normal(size=(5, 4)):
        sc = _S(np.zeros((1, 3), np.float32), np.full((1, 3), math.log(0.02), np.float32),
                q[None].astype(np.float32), np.zeros(1, np.float32), np.zeros((1, 1, 3), np.float32), 0)
        pr = O.project(sc, cam)
        s = math.exp(float(np.float32(math.log(0.02))))
        v = (f * s / 3.0) ** 2 + float(np.float32(0.3))
        np.testing.assert_allclose([pr["cov_xx"][0], pr["cov_yy"][0]], [v, v], rtol=1e-12)
        assert abs(pr["cov_xy"][0]) < 1e-12
        np.testing.assert_allclose([pr["mean_x"][0], pr["mean_y"][0]], [64.0, 64.0], atol=1e-12)


def test_colour_opacity_and_D():
    sc = rand_scene(64, 5, deg=3)
    cam = W.look_at((0.5, -4.0, 0.7), (0, 0, 0), 64, 48)
    pr = O.project(sc, cam)
    o = O.camera_center(cam)
    mu = sc.means.astype(np.float64)
    d = (mu - o) / np.linalg.norm(mu - o, axis=1, keepdims=True)
    Y = np.stack([real_sh_scipy(l, m, d) for l in range(4) for m in range(-l, l + 1)], axis=1)
    raw = np.einsum("nk,nkc->nc", Y, sc.sh.astype(np.float64)) + 0.5
    np.testing.assert_allclose(np.stack([pr["raw_r"], pr["raw_g"], pr["raw_b"]], 1), raw, atol=1e-12)
    np.testing.assert_allclose(np.stack([pr["r"], pr["g"], pr["b"]], 1), np.maximum(raw, 0), atol=1e-12)
    np.testing.assert_allclose(pr["alpha"], sps.expit(sc.opacity_logits.astype(np.float64)), rtol=1e-14)
    np.testing.assert_allclose(pr["D"], 3 * np.exp(sc.log_scales.astype(np.float64)).max(1), rtol=1e-14)


# --------------------------------------------------------------------------- Eq. 2 closed forms
def _iso_splat(z_world, scale, logit, dc, x=0.0, y=0.0):
    return (np.array([x, y, z_world], np.float32), np.full(3, math.log(scale), np.float32),
            np.array([1, 0, 0, 0], np.float32), np.float32(logit), np.array(dc, np.float32))


def _scene_of(splats):
    m, ls, q, lg, dc = zip(*splats)
    return _S(np.stack(m), np.stack(ls), np.stack(q), np.array(lg, np.float32), np.stack(dc)[:, None, :], 0)


def _closed_form_sigma(cam, mu_world, scale, logit, tm=3.0):
    """sigma and the contribution mask of one isotropic splat straight from Eq. 1-2."""
    f = float(np.float32(cam.fx))
    z = mu_world[2] + 3.0
    s = math.exp(float(np.float32(math.log(scale))))
    v = (f * s / z) ** 2 + float(np.float32(0.3))
    px, py = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    mx = f * mu_world[0] / z + 64.0
    my = f * mu_world[1] / z + 64.0
    r2 = (px - mx) ** 2 + (py - my) ** 2
    d2 = r2 / v
    alpha = 1 / (1 + math.exp(-float(np.float32(logit))))
    sigma = np.minimum(float(np.float32(0.99)), alpha * np.exp(-0.5 * d2))
    ok = (d2 <= tm * tm) & (z * z * r2 / (f * f) <= (tm * s) ** 2) & (sigma >= float(np.float32(1 / 255)))
    return np.where(ok, sigma, 0.0).reshape(-1)


def test_single_splat_closed_form():
    cam = W.axis_camera((0.0, 0.0, -3.0), 128, 128)
    sc = _scene_of([_iso_splat(0.0, 0.05, 1.3, [0.4, 0.2, 0.9])])
    out = O.render(sc, cam)
    sig = _closed_form_sigma(cam, (0.0, 0.0, 0.0), 0.05, 1.3)
    c0 = 0.5 / math.sqrt(math.pi)
    rgb = np.array([c0 * float(np.float32(v)) + 0.5 for v in (0.4, 0.2, 0.9)])
    np.testing.assert_allclose(out["C"], sig[:, None] * rgb[None], atol=1e-14)
    np.testing.assert_allclose(out["T"], 1 - sig, atol=1e-14)
    assert (sig > 0).sum() > 50


def test_two_splats_depth_order_closed_form():
    """C = c1 s1 + c2 s2 (1 - s1) with splat 1 the nearer one, whatever the index order."""
    cam = W.axis_camera((0.0, 0.0, -3.0), 128, 128)
    far = _iso_splat(1.0, 0.09, 0.5, [0.9, 0.1, 0.1])   # both on the optical axis, where the
    near = _iso_splat(0.0, 0.04, 1.0, [0.1, 0.8, 0.3])  # projected covariance is isotropic
    sc = _scene_of([far, near])           # the farther splat has the lower index
    out = O.render(sc, cam)
    s_far = _closed_form_sigma(cam, (0.0, 0.0, 1.0), 0.09, 0.5)
    s_near = _closed_form_sigma(cam, (0.0, 0.0, 0.0), 0.04, 1.0)
    c0 = 0.5 / math.sqrt(math.pi)
    c_far = np.array([c0 * float(np.float32(v)) + 0.5 for v in (0.9, 0.1, 0.1)])
    c_near = np.array([c0 * float(np.float32(v)) + 0.5 for v in (0.1, 0.8, 0.3)])
    expect = s_near[:, None] * c_near + (s_far * (1 - s_near))[:, None] * c_far
    np.testing.assert_allclose(out["C"], expect, atol=1e-14)
    np.testing.assert_allclose(out["T"], (1 - s_near) * (1 - s_far), atol=1e-14)
    both = (s_far > 0) & (s_near > 0)
    assert both.sum() > 50


def test_white_splats_colour_plus_transmittance_is_one():
    sc = rand_scene(300, 7)
    c0 = 0.5 / math.sqrt(math.pi)
    sc.sh = np.full_like(sc.sh, 0.5 / c0, dtype=np.float64)
    cam = W.look_at((0.3, -3.5, 0.4), (0, 0, 0), 48, 40)
    out = O.render(sc, cam)
    for c in range(3):
        np.testing.assert_allclose(out["C"][:, c] + out["T"], 1.0, atol=1e-12)
    assert (out["T"] < 0.5).sum() > 50


def _concat(a, b):
    return _S(*(np.concatenate([x, y]) for x, y in zip(
        (a.means, a.log_scales, a.quats, a.opacity_logits, a.sh),
        (b.means, b.log_scales, b.quats, b.opacity_logits, b.sh))), a.sh_degree)


def test_transmittance_monotone_when_splats_are_added():
    base = rand_scene(200, 11)
    extra = rand_scene(200, 12)
    more = _concat(base, extra)          # the same 200 splats plus 200 more
    cam = W.look_at((0.0, -3.0, 0.5), (0, 0, 0), 40, 40)
    t1 = O.render(base, cam)["T"]
    t2 = O.render(more, cam)["T"]
    assert np.all(t2 <= t1 + 1e-15)
    assert np.all((t1 >= 0) & (t1 <= 1))
    assert (t2 < t1 - 1e-3).sum() > 20
    extra.opacity_logits = np.full_like(extra.opacity_logits, -40.0)   # alpha ~ 4e-18 < alpha_min
    np.testing.assert_array_equal(O.render(_concat(base, extra), cam)["T"], t1)


def test_bbox_prefilter_equals_brute_force():
    sc = rand_scene(500, 13, log_scale=(-3.0, 0.6), deg=3)
    cam = W.look_at((1.0, -3.0, 0.5), (0, 0, 0), 40, 32)
    a = O.render(sc, cam)
    b = O.render(sc, cam, brute=True)
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["ncontrib"], b["ncontrib"])


# --------------------------------------------------------------------------- Eq. 3-6 == Eq. 2
def _random_tree(L, r, extent=1.0):
    K = 1 << L
    axis = r.integers(0, 3, K - 1).astype(np.int32)
    split = r.uniform(-0.6 * extent, 0.6 * extent, K - 1).astype(np.float32)
    return axis, split


@pytest.mark.parametrize("L", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hierarchical_equals_flat_random_trees(L, seed):
    """The equivalence derived in the appendix: Eq. 5 over Eq. 3-4 reproduces Eq. 2 for any
    convex partition, here random axis-aligned trees and cameras inside and outside."""
    r = np.random.default_rng(100 + seed)
    sc = rand_scene(96, seed, log_scale=(-2.2, 0.4), deg=2 if seed else 0)
    axis, split = _random_tree(L, r)
    eye = (0.2, -0.1, 0.1) if seed == 2 else (0.5, -3.0, 0.8)
    tgt = (0.0, 1.0, 0.0) if seed == 2 else (0, 0, 0)
    cam = W.look_at(eye, tgt, 32, 32)
    flat = O.render(sc, cam)
    hier = O.render(sc, cam, hier=True, L=L, axis=axis, split=split)
    np.testing.assert_allclose(hier["C"], flat["C"], atol=1e-12)
    np.testing.assert_allclose(hier["T"], flat["T"], atol=1e-12)
    assert flat["ncontrib"].sum() > 200
    if L == 0:
        np.testing.assert_allclose(hier["partC"][:, 0], flat["C"], atol=1e-15)
        np.testing.assert_allclose(hier["partT"][:, 0], flat["T"], atol=1e-15)
    else:
        # the partition really splits the work: more than one subset is non-trivial
        nontrivial = (hier["partT"] < 1).any(axis=0)
        assert nontrivial.sum() >= 2


def test_kd_tree_hierarchical_equals_flat():
    wl = W.tiny()
    axis, split = O.kd_partition(wl.scene.means, 3)
    sub = wl.scene
    flat = O.render(sub, wl.cameras[0])
    hier = O.render(sub, wl.cameras[0], hier=True, L=3, axis=axis, split=split)
    np.testing.assert_allclose(hier["C"], flat["C"], atol=1e-12)


def test_validity_optical_axis_on_dividing_plane():
    """Sec. 4 validity test: with the optical axis on the plane x = s every ray stays on one
    side, so each partial image is exactly (C, T) = (0, 1) on the other half."""
    sc = rand_scene(400, 21, log_scale=(-2.5, 0.4))
    s = np.float32(0.125)
    cam = W.axis_camera((float(s), 0.1, -3.0), 32, 24)
    out = O.render(sc, cam, hier=True, L=1, axis=np.array([0], np.int32), split=np.array([s], np.float32))
    px = np.arange(32 * 24) % 32
    left, right = px < 16, px >= 16
    assert np.all(out["partC"][left, 1] == 0) and np.all(out["partT"][left, 1] == 1)
    assert np.all(out["partC"][right, 0] == 0) and np.all(out["partT"][right, 0] == 1)
    assert (out["partT"][left, 0] < 1).sum() > 20 and (out["partT"][right, 1] < 1).sum() > 20
    flat = O.render(sc, cam)
    np.testing.assert_allclose(out["C"], flat["C"], atol=1e-12)


def test_straddling_splat_counted_once():
    """Appendix figure on boundary primitives: a splat crossing the dividing plane is in both
    subsets, but each ray takes its contribution from exactly one of them."""
    cam = W.axis_camera((0.03, 0.0, -3.0), 64, 64)
    sc = _scene_of([_iso_splat(0.0, 0.08, 2.0, [0.7, 0.3, 0.5])])
    axis, split = np.array([0], np.int32), np.array([0.0], np.float32)
    offs, idx, _ = O.subsets(sc.means, sc.log_scales, 1, axis, split)
    assert list(offs) == [0, 1, 2] and list(idx) == [0, 0]
    out = O.render(sc, cam, hier=True, L=1, axis=axis, split=split)
    flat = O.render(sc, cam)
    np.testing.assert_allclose(out["C"], flat["C"], atol=1e-15)
    touched = out["partT"] < 1
    assert np.all(touched.sum(axis=1) <= 1)
    assert touched[:, 0].sum() > 20 and touched[:, 1].sum() > 20


# --------------------------------------------------------------------------- Sec. 3.3 KD tree
def _read_kd_golden():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "kd_splits.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("case"):
            cur = {"name": line.split()[1], "pts": []}
            cases.append(cur)
        elif line.startswith("L "):
            cur["L"] = int(line.split()[1])
        elif line.startswith("splits"):
            cur["splits"] = [float(v) for v in line.split()[1:]]
        else:
            cur["pts"].append([float(v) for v in line.split()])
    return cases


@pytest.mark.parametrize("case", _read_kd_golden(), ids=lambda c: c["name"])
def test_kd_golden(case):
    pts = np.array(case["pts"], np.float32)
    axis, split = O.kd_partition(pts, case["L"])
    np.testing.assert_array_equal(split, np.array(case["splits"], np.float32))
    np.testing.assert_array_equal(axis, [(int(math.log2(j + 1))) % 3 for j in range(len(split))])


def test_kd_balance_and_sides():
    r = np.random.default_rng(4)
    for n, L in [(10_000, 4), (777, 3), (5, 2)]:
        pts = r.normal(size=(n, 3)).astype(np.float32)
        axis, split = O.kd_partition(pts, L)
        node = np.zeros(n, np.int64)
        for d in range(L):
            for j in range((1 << d) - 1, (1 << (d + 1)) - 1):
                members = node == j
                left = members & (pts[:, axis[j]] < split[j])
                assert abs(int(left.sum()) - int((members & ~left).sum())) <= 1
            node = np.where(pts[np.arange(n), axis[node]] < split[node], 2 * node + 1, 2 * node + 2)
        lo, hi = O.leaf_boxes(L, axis, split)
        leaf = node - ((1 << L) - 1)
        p64 = pts.astype(np.float64)
        assert np.all((p64 >= lo[leaf]) & (p64 < hi[leaf]))


def test_subsets_equal_dilated_boxes():
    """N_k by the plane rule equals {i : mu_i within the box S_k dilated by D_i}, and every
    splat whose centre lies in S_k is in N_k."""
    sc = rand_scene(3000, 8, log_scale=(-2.5, 0.7))
    L = 3
    axis, split = O.kd_partition(sc.means, L)
    offs, idx, _ = O.subsets(sc.means, sc.log_scales, L, axis, split)
    lo, hi = O.leaf_boxes(L, axis, split)
    mu = sc.means.astype(np.float64)
    D = 3 * np.exp(sc.log_scales.astype(np.float64)).max(1)
    for k in range(1 << L):
        expect = np.nonzero(np.all((mu + D[:, None] >= lo[k]) & (mu - D[:, None] < hi[k]), axis=1))[0]
        np.testing.assert_array_equal(idx[offs[k]:offs[k + 1]], expect)
        inside = np.nonzero(np.all((mu >= lo[k]) & (mu < hi[k]), axis=1))[0]
        assert np.isin(inside, expect).all()
    assert offs[-1] > mu.shape[0]          # overlap: some splats belong to several subsets


def test_ray_order_matches_dense_sampling():
    r = np.random.default_rng(6)
    pts = r.normal(size=(2000, 3)).astype(np.float32)
    L = 4
    axis, split = O.kd_partition(pts, L)
    lo, hi = O.leaf_boxes(L, axis, split)
    for _ in range(25):
        o = r.normal(size=3) * 1.5
        d = r.normal(size=3)
        order, nc = O.ray_order(L, axis, split, o, d)
        t = np.arange(0, 12, 2e-4)
        x = o[None] + t[:, None] * d[None]
        inside = np.all((x[:, None, :] >= lo[None]) & (x[:, None, :] < hi[None]), axis=2)
        leaf = np.argmax(inside, axis=1)
        seen = []
        for k in leaf:
            if not seen or seen[-1] != k:
                seen.append(int(k))
        assert len(set(seen)) == len(seen)
        assert list(order[:len(seen)]) == seen
        assert sorted(order.tolist()) == list(range(1 << L))


# --------------------------------------------------------------------------- foot reading of x_i
# The comparison reading of Sec. 3.2: x_i is the foot of the perpendicular from the splat
# centre onto the pixel ray and each ray's contributors are ordered by its ray parameter.
FOOT = O.Opts(foot=True)


def _ray(cam, px, py):
    """Camera centre and unit world direction of the ray through pixel centre (px, py)."""
    V = np.asarray(cam.viewmat, np.float32).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    d = V[:3, :3].T @ np.array([(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0])
    return -V[:3, :3].T @ V[:3, 3], d / np.linalg.norm(d)


def _closest_on_ray(o, d, mu):
    """(t, distance) of the point of the ray o + t d nearest to mu, by a bounded scalar
    minimisation of the distance (not the projection formula)."""
    from scipy.optimize import minimize_scalar
    f = lambda t: float(np.sum((o + t * d - mu) ** 2))
    span = float(np.linalg.norm(mu - o)) * 2 + 1.0
    res = minimize_scalar(f, bounds=(-span, span), method="bounded", options={"xatol": 1e-12})
    return res.x, math.sqrt(max(res.fun, 0.0))


def test_foot_equals_depth_plane_on_a_ray_through_every_centre():
    """Centres on one pixel's ray: there the foot is the centre itself, as is the ray point
    at the centre's depth, so both readings give that pixel the same colour."""
    cam = W.look_at((0.4, -3.0, 0.6), (0, 0, 0), 48, 40)
    px, py = 30, 13
    o, d = _ray(cam, px, py)
    lam = np.array([2.2, 2.9, 3.1, 3.6, 4.4])
    splats = [(np.float32(o + l * d).astype(np.float32), np.full(3, -2.6, np.float32),
               np.array([0.9, 0.1, -0.3, 0.2], np.float32), np.float32(0.4 + 0.3 * j),
               np.array([0.2 * j, 0.9 - 0.15 * j, 0.5], np.float32)) for j, l in enumerate(lam)]
    sc = _scene_of(splats[::-1])
    pix = [py * cam.width + px]
    a = O.render(sc, cam, pix=pix)
    b = O.render(sc, cam, FOOT, pix=pix)
    assert a["ncontrib"][0] == len(lam) and b["ncontrib"][0] == len(lam)
    np.testing.assert_allclose(b["C"], a["C"], atol=1e-12)
    np.testing.assert_allclose(b["T"], a["T"], atol=1e-12)


def test_foot_ball_region_matches_minimised_distance():
    """Small, opaque, isotropic splats whose screen ellipse (with the dilation) holds the
    ball: a pixel counts a splat iff the ray passes within D of its centre, the distance
    found by minimising along the ray.  The depth-plane reading accepts fewer pixels."""
    cam = W.axis_camera((0.0, 0.0, -3.0), 64, 64)
    r = np.random.default_rng(3)
    n = 10
    xy = r.uniform(-1.3, 1.3, (n, 2))
    splats = [_iso_splat(float(r.uniform(-0.3, 0.3)), 0.05, 6.0, [0.3, 0.3, 0.3], x=float(a), y=float(b))
              for a, b in xy]
    sc = _scene_of(splats)
    foot = O.render(sc, cam, FOOT)
    plane = O.render(sc, cam)
    proj = O.project(sc, cam)
    D = proj["D"]
    expect = np.zeros(cam.width * cam.height, np.int64)
    near_edge = np.zeros(cam.width * cam.height, bool)
    for q in range(cam.width * cam.height):
        px, py = q % cam.width, q // cam.width
        o, d = _ray(cam, px, py)
        for i in range(n):
            dx = px + 0.5 - proj["mean_x"][i]
            dy = py + 0.5 - proj["mean_y"][i]
            if dx * dx + dy * dy > 400:            # far outside every footprint
                continue
            _, dist = _closest_on_ray(o, d, sc.means[i].astype(np.float64))
            if abs(dist - D[i]) < 1e-6 * D[i]:
                near_edge[q] = True
            if dist <= D[i]:
                expect[q] += 1
                # precondition: the ellipse d^2 <= 9 holds every pixel of the ball
                d2 = proj["conic_a"][i] * dx * dx + 2 * proj["conic_b"][i] * dx * dy + proj["conic_c"][i] * dy * dy
                assert d2 <= 9.0 * (1 - 1e-3)
    ok = ~near_edge
    np.testing.assert_array_equal(foot["ncontrib"][ok], expect[ok])
    assert np.all(foot["ncontrib"] >= plane["ncontrib"])
    assert (foot["ncontrib"] > plane["ncontrib"]).sum() >= 10
    assert expect.sum() > 200


def test_foot_order_follows_the_ray_parameter():
    """Two overlapping splats whose order along the ray flips inside the overlap: the foot
    reading composites them in the order of the minimised ray parameter, the depth-plane
    reading always puts the nearer centre first."""
    cam = W.axis_camera((0.0, 0.0, -3.0), 64, 64)
    A = _iso_splat(0.0, 0.2, 2.0, [0.9, 0.1, 0.1], x=-0.3)
    B = _iso_splat(0.02, 0.2, 2.0, [0.1, 0.1, 0.9], x=0.3)
    both = O.render(_scene_of([A, B]), cam, FOOT)
    sA = 1 - O.render(_scene_of([A]), cam, FOOT)["T"]
    sB = 1 - O.render(_scene_of([B]), cam, FOOT)["T"]
    c0 = 0.5 / math.sqrt(math.pi)
    cA = np.array([c0 * float(np.float32(v)) + 0.5 for v in (0.9, 0.1, 0.1)])
    cB = np.array([c0 * float(np.float32(v)) + 0.5 for v in (0.1, 0.1, 0.9)])
    flips = 0
    for q in np.nonzero((sA > 0.02) & (sB > 0.02))[0]:
        o, d = _ray(cam, q % cam.width, q // cam.width)
        tA, _ = _closest_on_ray(o, d, np.array(A[0], np.float64))
        tB, _ = _closest_on_ray(o, d, np.array(B[0], np.float64))
        if abs(tA - tB) < 1e-6:
            continue
        if tA < tB:
            expect = sA[q] * cA + sB[q] * (1 - sA[q]) * cB
        else:
            expect = sB[q] * cB + sA[q] * (1 - sB[q]) * cA
            flips += 1
        np.testing.assert_allclose(both["C"][q], expect, atol=1e-12)
    assert flips >= 5
    plane = O.render(_scene_of([A, B]), cam)
    assert np.abs(plane["C"] - both["C"]).max() > 1e-3


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_foot_hierarchical_equals_flat(L, seed):
    """The appendix's equivalence holds for the foot reading too: the foot lies on the ray,
    so every convex subspace holds one interval of the ray parameter."""
    r = np.random.default_rng(200 + seed)
    sc = rand_scene(96, 40 + seed, log_scale=(-2.0, 0.4), deg=2 if seed else 0)
    axis, split = _random_tree(L, r)
    cam = W.look_at((0.6, -2.6, 0.9), (0, 0, 0), 32, 32)
    flat = O.render(sc, cam, FOOT)
    hier = O.render(sc, cam, FOOT, hier=True, L=L, axis=axis, split=split)
    np.testing.assert_allclose(hier["C"], flat["C"], atol=1e-12)
    np.testing.assert_allclose(hier["T"], flat["T"], atol=1e-12)
    assert flat["ncontrib"].sum() > 200
    assert ((hier["partT"] < 1).any(axis=0)).sum() >= 2
    assert np.abs(flat["C"] - O.render(sc, cam)["C"]).max() > 1e-4   # the readings differ here


# --------------------------------------------------------------------------- adjoint vs FD
def _loss(sc, cam, w, opts):
    return float(np.sum(O.render(sc, cam, opts)["C"] * w))


@pytest.mark.parametrize("deg,foot", [(0, False), (3, False), (3, True)])
def test_adjoint_matches_finite_differences(deg, foot):
    """Hand-written reverse mode vs central differences of the FP64 forward for L = <w, C>,
    every parameter of every splat; perturbations that change the set of contributing
    pairs or their order are skipped.  foot: the same under the perpendicular-foot reading
    of x_i (its own contributors and per-ray order)."""
    sc0 = rand_scene(16, 30 + deg, extent=0.6, log_scale=(-2.0, 0.3), deg=deg).copy()
    cam = W.look_at((0.4, -2.5, 0.6), (0, 0, 0), 20, 16)
    opts = O.Opts(bg=(0.1, 0.2, 0.3), foot=foot)
    w = np.random.default_rng(1).uniform(-1, 1, (cam.width * cam.height, 3))
    adj = O.adjoint(sc0, cam, w, opts)
    sig0 = O.pair_signature(sc0, cam, opts)
    names = [("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"),
             ("opacity_logits", "opacity_logits"), ("sh", "sh")]
    checked = skipped = 0
    for attr, key in names:
        arr = getattr(sc0, attr)
        g = adj[key]
        scale = max(np.abs(g).max(), 1e-12)
        for flat_i in range(arr.size):
            x0 = arr.reshape(-1)[flat_i]
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            ok = True
            for sgn in (1, -1):
                sc = sc0.copy()
                getattr(sc, attr).reshape(-1)[flat_i] = x0 + sgn * h
                if O.pair_signature(sc, cam, opts) != sig0:
                    ok = False
                    break
                vals.append(_loss(sc, cam, w, opts))
            if not ok:
                skipped += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g.reshape(-1)[flat_i]) <= 2e-6 * scale + 1e-7 * abs(fd), (attr, flat_i, fd, g.reshape(-1)[flat_i])
            checked += 1
    assert checked > 0.95 * (checked + skipped)
    assert np.abs(adj["means"]).max() > 0 and np.abs(adj["sh"]).max() > 0
    if foot:   # the reading matters in this scene: its gradients are not the depth plane's
        other = O.adjoint(sc0, cam, w, O.Opts(bg=(0.1, 0.2, 0.3)))
        assert np.abs(other["means"] - adj["means"]).max() > 1e-3 * np.abs(adj["means"]).max()


# --------------------------------------------------------------------------- Eq. 5 merge
def _rand_partials(K, P, seed):
    r = np.random.default_rng(seed)
    T = r.uniform(0.05, 1.0, (K, P))
    C = r.uniform(0, 1, (K, 3, P)) * (1 - T)[:, None]
    return C, T


def test_merge_single_subset_identity_and_trivial_subsets():
    C, T = _rand_partials(1, 50, 0)
    mC, mT = O.merge(C, T, [0])
    np.testing.assert_array_equal(mC, C[0])
    np.testing.assert_array_equal(mT, T[0])
    C4, T4 = _rand_partials(4, 50, 1)
    base, baseT = O.merge(C4, T4, [2, 0, 3, 1])
    Cx = np.concatenate([C4, np.zeros((1, 3, 50))])
    Tx = np.concatenate([T4, np.ones((1, 50))])
    for pos in range(5):
        order = [2, 0, 3, 1]
        order.insert(pos, 4)
        got, gotT = O.merge(Cx, Tx, order)
        np.testing.assert_allclose(got, base, atol=1e-15)
        np.testing.assert_allclose(gotT, baseT, atol=1e-15)


def test_merge_associative():
    C, T = _rand_partials(6, 40, 2)
    order = [3, 1, 5, 0, 2, 4]
    full, fullT = O.merge(C, T, order, bg=(0.2, 0.1, 0.4))
    for j in range(1, 6):
        fC, fT = O.merge(C, T, order[:j])
        bC, bT = O.merge(C, T, order[j:], bg=(0.2, 0.1, 0.4))
        np.testing.assert_allclose(fC + fT * bC, full, atol=1e-14)
        np.testing.assert_allclose(fT * bT, fullT, atol=1e-15)


def test_merge_backward_matches_fd():
    K, P = 5, 7
    C, T = _rand_partials(K, P, 3)
    order = np.array([4, 2, 0, 1, 3])
    r = np.random.default_rng(4)
    g = r.uniform(-1, 1, (3, P))
    gT = r.uniform(-1, 1, P)
    bg = (0.3, 0.6, 0.1)
    dC, dT = O.merge_backward(C, T, order, g, gT, bg=bg)

    def loss(C_, T_):
        mc, mt = O.merge(C_, T_, order, bg=bg)
        return float(np.sum(mc * g) + np.sum(mt * gT))

    h = 1e-6
    for idx in np.ndindex(C.shape):
        Cp, Cm = C.copy(), C.copy()
        Cp[idx] += h
        Cm[idx] -= h
        assert abs((loss(Cp, T) - loss(Cm, T)) / (2 * h) - dC[idx]) < 1e-8
    for idx in np.ndindex(T.shape):
        Tp, Tm = T.copy(), T.copy()
        Tp[idx] += h
        Tm[idx] -= h
        assert abs((loss(C, Tp) - loss(C, Tm)) / (2 * h) - dT[idx]) < 1e-8


# --------------------------------------------------------------------------- Adam
def test_adam_closed_form_steps():
    p0 = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -0.2, 0.0])
    p1, m1, v1 = O.adam_step(p0, g1, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * sign(g) (0 where g = 0)
    np.testing.assert_allclose(p1, p0 - 0.01 * np.sign(g1), atol=1e-12)
    g2 = np.array([0.1, 0.4, -1.0])
    p2, m2, v2 = O.adam_step(p1, g2, m1, v1, 2, lr=0.01)
    m_hand = 0.9 * 0.1 * g1 + 0.1 * g2
    v_hand = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    np.testing.assert_allclose(m2, m_hand, rtol=1e-15)
    np.testing.assert_allclose(v2, v_hand, rtol=1e-15)
    upd = (m_hand / (1 - 0.81)) / (np.sqrt(v_hand / (1 - 0.999 ** 2)) + 1e-15)
    np.testing.assert_allclose(p2, p1 - 0.01 * upd, rtol=1e-14)


def test_position_lr_schedule():
    assert O.position_lr(0, 60000) == pytest.approx(1.6e-4, rel=1e-14)
    assert O.position_lr(60000, 60000) == pytest.approx(1.6e-6, rel=1e-14)
    assert O.position_lr(30000, 60000) == pytest.approx(1.6e-5, rel=1e-12)
    assert O.position_lr(120000, 60000) == pytest.approx(1.6e-6, rel=1e-14)
