"""Oracle pins of the Gaussian splatting forward renderer (Sec. 3.2.1 formula,
Sec. 3.5 rendering): closed forms for one and two Gaussians, the perspective
projection of the covariance against a finite-difference Jacobian, the 3-sigma
cutoff, the transmittance floor, and invariance under a joint rotation of scene
and camera."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def cam(w=32, h=24, f=40.0, R=np.eye(3), t=(0, 0, 0), bg=(0.1, 0.2, 0.3)):
    return O.make_camera(R, t, f, f, w / 2, h / 2, w, h, 0.01, bg)


def pixel_centres(c):
    py, px = np.mgrid[0:c.height, 0:c.width]
    return px + 0.5, py + 0.5


def test_one_gaussian_on_the_axis():
    c = cam()
    z, s, sig = 4.0, 0.2, 0.8
    x = np.array([[0.0, 0.0, z]])
    A = (s * s * np.eye(3))[None]
    col = np.array([[1.0, 0.5, 0.25]])
    rgb, T = O.splat_render(x, [sig], A, col, c)
    pu, pv = pixel_centres(c)
    r2 = (pu - c.cx) ** 2 + (pv - c.cy) ** 2
    ss = (c.fx * s / z) ** 2                      # projected variance (pixels^2)
    md = r2 / ss
    a = np.minimum(0.99, sig * np.exp(-0.5 * md))
    a = np.where((md <= 9.0) & (a >= 1 / 255), a, 0.0)
    bg = np.array(c.bg)
    exp = a[..., None] * col[0] + (1 - a)[..., None] * bg
    assert np.allclose(rgb, exp, atol=1e-12)
    assert np.allclose(T, 1 - a, atol=1e-12)


def test_two_gaussians_composite_front_to_back_by_depth():
    c = cam()
    A = np.stack([0.04 * np.eye(3)] * 2)
    cols = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    # index 0 is behind index 1: depth decides
    x = np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 4.0]])
    rgb, T = O.splat_render(x, [0.7, 0.6], A, cols, c)
    pu, pv = pixel_centres(c)
    r2 = (pu - c.cx) ** 2 + (pv - c.cy) ** 2
    def alpha(z, sig):
        md = r2 / (c.fx * 0.2 / z) ** 2
        a = np.minimum(0.99, sig * np.exp(-0.5 * md))
        return np.where((md <= 9.0) & (a >= 1 / 255), a, 0.0)
    a1, a0 = alpha(4.0, 0.6), alpha(5.0, 0.7)
    exp = a1[..., None] * cols[1] + ((1 - a1) * a0)[..., None] * cols[0] + ((1 - a1) * (1 - a0))[..., None] * np.array(c.bg)
    assert np.allclose(rgb, exp, atol=1e-12)


def test_perspective_covariance_matches_a_finite_difference_jacobian():
    th = 0.3
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    c = cam(64, 48, 55.0, R=R, t=(0.1, -0.2, 3.0))
    x = np.array([0.4, 0.3, 1.0])
    L = np.array([[0.2, 0.0, 0.0], [0.05, 0.15, 0.0], [0.02, -0.03, 0.1]])
    A = L @ L.T

    def proj(p):
        q = R @ p + np.array([0.1, -0.2, 3.0])
        return np.array([c.fx * q[0] / q[2] + c.cx, c.fy * q[1] / q[2] + c.cy])

    h = 1e-6
    J = np.stack([(proj(x + h * e) - proj(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
    S = J @ A @ J.T
    m = proj(x)
    rgb, T = O.splat_render(x[None], [0.9], A[None], np.ones((1, 3)), c)
    pu, pv = pixel_centres(c)
    d = np.stack([pu - m[0], pv - m[1]], -1)
    md = np.einsum("...i,ij,...j->...", d, np.linalg.inv(S), d)
    a = np.minimum(0.99, 0.9 * np.exp(-0.5 * md))
    a = np.where((md <= 9.0) & (a >= 1 / 255), a, 0.0)
    assert np.allclose(1 - T, a, atol=1e-7)


def test_cutoff_floor_and_culling():
    c = cam(24, 24, 30.0, bg=(0, 0, 0))
    rng = np.random.default_rng(0)
    n = 60
    x = np.column_stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(2, 3, n)])
    A = np.stack([0.3 ** 2 * np.eye(3)] * n)
    rgb, T = O.splat_render(x, np.full(n, 0.99), A, np.ones((n, 3)), c)
    assert T.min() >= 1e-4 * (1 - 0.99) and T.min() < 1e-2   # the floor stops the walk
    # a Gaussian behind the camera contributes nothing
    rgb2, T2 = O.splat_render(np.array([[0, 0, -2.0]]), [0.9], A[:1], np.ones((1, 3)), c)
    assert np.all(T2 == 1.0) and np.all(rgb2 == 0.0)
    # pixels beyond the 3-sigma ellipse see nothing
    rgb3, T3 = O.splat_render(np.array([[0, 0, 2.0]]), [0.99], (0.01 ** 2 * np.eye(3))[None], np.ones((1, 3)), c)
    assert (T3 < 1).sum() <= 9


def test_joint_rotation_of_scene_and_camera_changes_nothing():
    rng = np.random.default_rng(3)
    n = 40
    x = np.column_stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(2, 4, n)])
    L = rng.standard_normal((n, 3, 3)) * 0.08
    A = L @ np.transpose(L, (0, 2, 1)) + 1e-3 * np.eye(3)
    col, op = rng.random((n, 3)), rng.uniform(0.2, 0.9, n)
    c = cam(40, 30, 45.0)
    rgb, T = O.splat_render(x, op, A, col, c)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    c2 = cam(40, 30, 45.0, R=Q.T)           # x_c = Q^T (Q x) = x
    rgb2, T2 = O.splat_render(x @ Q.T, op, Q @ A @ Q.T, col, c2)
    assert np.allclose(rgb, rgb2, atol=1e-9) and np.allclose(T, T2, atol=1e-9)


def test_walk_stops_before_the_gaussian_that_would_cross_the_floor():
    """One pixel on the axis, three Gaussians behind it with alphas 0.98, 0.99 and
    0.99 (opacities 0.98, 0.99 and 1.0, the last capped): after two, T = 0.02 *
    0.01 = 2e-4 is still above the 1e-4 floor, so both are composited; the third
    would take T to 2e-6, so the walk stops before it and it adds nothing."""
    c = cam(1, 1, 40.0, bg=(0.0, 0.0, 0.0))       # pixel centre (0.5, 0.5) = the axis
    x = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, 3.0], [0.0, 0.0, 4.0]])
    A = np.stack([0.2 ** 2 * np.eye(3)] * 3)
    cols = np.eye(3)
    rgb, T = O.splat_render(x, [0.98, 0.99, 1.0], A, cols, c)
    assert T[0, 0] == pytest.approx(0.02 * 0.01, rel=1e-12)
    assert rgb[0, 0, 0] == pytest.approx(0.98, rel=1e-12)
    assert rgb[0, 0, 1] == pytest.approx(0.02 * 0.99, rel=1e-12)
    assert rgb[0, 0, 2] == 0.0
    # without the third Gaussian in front of the floor, the first two are unchanged
    rgb2, T2 = O.splat_render(x[:2], [0.98, 0.99], A[:2], cols[:2], c)
    assert np.allclose(rgb2, rgb) and np.allclose(T2, T)


def test_alpha_threshold_of_one_over_255():
    """A Gaussian whose alpha at the pixel centre sits just below 1/255 leaves the
    pixel untouched; just above, it is composited."""
    c = cam(1, 1, 40.0, bg=(0.0, 0.0, 0.0))       # one pixel, centre on the axis
    A = (0.2 ** 2 * np.eye(3))[None]
    x = np.array([[0.0, 0.0, 2.0]])
    lo, hi = (1.0 / 255.0) * (1 - 1e-6), (1.0 / 255.0) * (1 + 1e-6)
    _, T_lo = O.splat_render(x, [lo], A, np.ones((1, 3)), c)
    rgb_hi, T_hi = O.splat_render(x, [hi], A, np.ones((1, 3)), c)
    assert T_lo[0, 0] == 1.0
    assert T_hi[0, 0] == pytest.approx(1.0 - hi, abs=1e-15) and rgb_hi[0, 0, 0] == pytest.approx(hi, abs=1e-15)
