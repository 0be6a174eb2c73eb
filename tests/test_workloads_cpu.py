"""The seeded input recipes hold what the design notes state about them: occupancy
of the blob and the sphere union, the inflow patch of the river scene, the blurred
fields' zero wall-normal faces, the Gaussian cloud's counts, positions, covariance
scales, opacities and colours, and the look-at camera's geometry; every recipe is
reproducible from its seed."""
import numpy as np
import pytest

from paper_2503_00868_gb300 import workloads as W


def test_blob_occupancy_and_seed():
    t, info = W.ellipsoid_blob(64, 64, 64, 0)
    assert abs(info["occupancy"] - 0.40) < 0.03
    assert info["occupancy"] == pytest.approx(float((t == W.LIQUID).mean()))
    assert np.array_equal(t, W.ellipsoid_blob(64, 64, 64, 0)[0])
    assert not np.array_equal(t, W.ellipsoid_blob(64, 64, 64, 1)[0])
    assert set(np.unique(t)) <= {W.AIR, W.LIQUID}


def test_sphere_union_occupancy_range():
    for seed in range(3):
        t, info = W.sphere_union(48, 48, 48, seed)
        assert 0.15 <= info["occupancy"] <= 0.50


def test_river_inflow_patch():
    nx, ny, nz = 30, 20, 26
    types, inflow, info = W.river_with_blob(nx, ny, nz, 0)
    assert inflow.shape == (nz, ny, nx + 1)
    k, j, i = np.nonzero(inflow)
    assert np.all(i == 0)                            # the x = 0 wall faces only
    assert np.all(types[k, j, 0] == W.LIQUID)        # of liquid cells
    assert np.all((j + 0.5) / ny <= 0.25 + 1e-12)    # below the 0.25 m layer


def test_blurred_fields_have_zero_wall_normal_faces():
    u, v, w = W.blurred_noise_mac(20, 18, 16, 3)
    assert np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    assert np.all(v[:, 0, :] == 0) and np.all(v[:, -1, :] == 0)
    assert np.all(w[0] == 0) and np.all(w[-1] == 0)
    assert float(np.abs(u[:, :, 1:-1]).max()) > 0


def test_gaussian_cloud_recipe():
    n = 32
    dx = 1.0 / n
    types, _ = W.ellipsoid_blob(n, n, n, 0)
    x, op, A, col = W.gaussian_cloud(types, dx, 5)
    k, j, i = np.nonzero(types == W.LIQUID)
    assert x.shape == (k.size, 3) and op.shape == (k.size,) and A.shape == (k.size, 3, 3)
    centres = (np.stack([i, j, k], axis=1) + 0.5) * dx
    assert np.all(np.abs(x - centres) <= 0.25 * dx + 1e-12)          # jitter of +-dx/4
    assert np.allclose(A, np.transpose(A, (0, 2, 1)))
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= (0.3 * dx) ** 2 * (1 - 1e-9) and ev.max() <= (0.9 * dx) ** 2 * (1 + 1e-9)
    assert op.min() >= 0.3 and op.max() <= 0.95
    assert col.min() >= 0.0 and col.max() <= 1.0


def test_look_at_camera():
    target = np.array([0.5, 0.2, 0.5])
    R, t, fx, fy, cx, cy = W.look_at(target, 1.6, 0.6, 0.35, 320, 240, fov_y=0.8)
    assert np.allclose(R @ R.T, np.eye(3)) and np.linalg.det(R) == pytest.approx(1.0)
    assert np.allclose(R @ target + t, [0.0, 0.0, 1.6])     # the target on the axis, 1.6 m ahead
    assert fx == fy == pytest.approx(120.0 / np.tan(0.4))
    assert (cx, cy) == (160.0, 120.0)
    up = R @ np.array([0.0, 1.0, 0.0])                       # world up points up in the image
    assert up[1] < 0.0
