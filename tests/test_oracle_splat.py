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


def test_near_threshold_flags_mark_exactly_the_ambiguous_pixels():
    """One isotropic Gaussian on the axis: sigma 0.1 at depth 2 seen with f = 40
    projects to a 2-pixel isotropic 2D Gaussian, so md = d^2 / 4 with d the pixel
    centre's distance to the mean in pixels. With the mean on a pixel corner
    (cx, cy = 20.5, 15.5) d^2 is an integer and md = 9 exactly at the four
    pixels 6 away along the axes: those, and only those, are flagged at rel 1e-3
    (alpha never reaches 1/255 before the cutoff, T stays above the floor). The
    flags change no value."""
    c = O.make_camera(np.eye(3), (0, 0, 0), 40.0, 40.0, 20.5, 15.5, 41, 31, 0.01, (0.1, 0.2, 0.3))
    x = np.array([[0.0, 0.0, 2.0]])
    A = (0.1 ** 2 * np.eye(3)).reshape(1, 9)
    op, col = np.array([0.9]), np.array([[0.3, 0.6, 0.9]])
    rgb, T = O.splat_render(x, op, A, col, c)
    rgb2, T2, near = O.splat_render(x, op, A, col, c, near_rel=1e-3)
    assert np.array_equal(rgb, rgb2) and np.array_equal(T, T2)
    py, px = np.nonzero(near)
    got = sorted(zip((px + 0.5 - 20.5).astype(int), (py + 0.5 - 15.5).astype(int)))
    assert got == [(-6, 0), (0, -6), (0, 6), (6, 0)]


def test_sh_basis_is_orthonormal_on_the_sphere():
    """The 16 real spherical harmonics of degree <= 3 integrate to the identity
    over the sphere: a Fibonacci lattice of 200 000 directions, each weighted
    4 pi / N, gives <Y_i, Y_j> to 1e-4. A wrong constant or a dropped term of any
    basis polynomial breaks this."""
    N = 200_000
    k = np.arange(N) + 0.5
    z = 1.0 - 2.0 * k / N
    phi = np.pi * (1.0 + 5.0 ** 0.5) * k
    r = np.sqrt(1.0 - z * z)
    dirs = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    Y = np.stack([O.sh_basis(3, d) for d in dirs[::50]])          # a coarse check of the call itself
    assert Y.shape == (N // 50, 16)
    # the full lattice through the same function, vectorised by rows of 1000
    G = np.zeros((16, 16))
    for s in range(0, N, 1000):
        Ys = np.stack([O.sh_basis(3, d) for d in dirs[s:s + 1000]])
        G += Ys.T @ Ys
    G *= 4.0 * np.pi / N
    np.testing.assert_allclose(G, np.eye(16), atol=1e-4)


def test_sh_sign_convention_along_the_axes():
    """The signs of the standard 3DGS evaluator: the degree-1 functions are
    -a y, a z, -a x (a = sqrt(3 / 4 pi))."""
    a = np.sqrt(3.0 / (4.0 * np.pi))
    np.testing.assert_allclose(O.sh_basis(1, [1, 0, 0]), [0.5 / np.sqrt(np.pi), 0, 0, -a], atol=1e-15)
    np.testing.assert_allclose(O.sh_basis(1, [0, 1, 0]), [0.5 / np.sqrt(np.pi), -a, 0, 0], atol=1e-15)
    np.testing.assert_allclose(O.sh_basis(1, [0, 0, 1]), [0.5 / np.sqrt(np.pi), 0, a, 0], atol=1e-15)


def test_sh_degree_zero_is_the_rgb_colour_and_degree_one_turns_with_the_view():
    """Degree 0 with coefficient (c - 1/2) / Y_0 renders exactly as the RGB colour
    c. One Gaussian on the optical axis with only the z coefficient of degree 1
    set: its colour is max(0, 1/2 + k a d_z) with d the direction from the camera
    centre to the mean, so the centre pixel is alpha colour + (1 - alpha) bg, and a
    camera on the other side (d_z = -1) sees 1/2 - k a."""
    rng = np.random.default_rng(4)
    n = 40
    x = np.column_stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.5, 3.0, n)])
    A = np.stack([0.03 ** 2 * np.eye(3)] * n).reshape(n, 9)
    op, col = rng.uniform(0.3, 0.9, n), rng.random((n, 3))
    c = cam()
    y0 = 0.5 / np.sqrt(np.pi)
    sh0 = ((col - 0.5) / y0).reshape(n, 1, 3)
    a_rgb, a_T = O.splat_render(x, op, A, col, c)
    b_rgb, b_T = O.splat_render_sh(x, op, A, sh0, 0, c)
    np.testing.assert_allclose(b_rgb, a_rgb, atol=1e-13)
    np.testing.assert_allclose(b_T, a_T, atol=1e-15)
    # one Gaussian on the axis, 2 m in front of the camera
    aa = np.sqrt(3.0 / (4.0 * np.pi))
    kz = np.array([0.3, -0.2, 0.6])
    sh = np.zeros((1, 4, 3))
    sh[0, 2] = kz
    xg = np.array([[0.0, 0.0, 2.0]])
    Ag = (0.05 ** 2 * np.eye(3)).reshape(1, 9)
    c1 = O.make_camera(np.eye(3), (0, 0, 0), 40.0, 40.0, 16.0, 12.0, 32, 24, 0.01, (0.1, 0.2, 0.3))
    rgb, T = O.splat_render_sh(xg, np.array([0.8]), Ag, sh, 1, c1)
    # pixel (15, 11) has its centre half a pixel from the mean in x and y
    s2 = (40.0 * 0.05 / 2.0) ** 2
    alpha = 0.8 * np.exp(-0.5 * (0.25 + 0.25) / s2)
    expect = alpha * np.maximum(0.0, 0.5 + kz * aa) + (1.0 - alpha) * np.array([0.1, 0.2, 0.3])
    np.testing.assert_allclose(rgb[11, 15], expect, rtol=1e-12)
    # the camera behind the Gaussian looking back along -z: R = diag(-1, 1, -1), centre at z = 4
    Rb = np.diag([-1.0, 1.0, -1.0])
    c2 = O.make_camera(Rb, -Rb @ np.array([0.0, 0.0, 4.0]), 40.0, 40.0, 16.0, 12.0, 32, 24, 0.01, (0.1, 0.2, 0.3))
    rgb2, _ = O.splat_render_sh(xg, np.array([0.8]), Ag, sh, 1, c2)
    expect2 = alpha * np.maximum(0.0, 0.5 - kz * aa) + (1.0 - alpha) * np.array([0.1, 0.2, 0.3])
    np.testing.assert_allclose(rgb2[11, 16], expect2, rtol=1e-12)
