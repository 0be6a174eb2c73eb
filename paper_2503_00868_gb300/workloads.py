"""Seeded synthetic inputs shaped like the paper's scenes.

This module only draws inputs: masks and velocity fields. It holds none of the
fluid step's arithmetic, so both the CUDA path and the FP64 oracle can be fed
from it without sharing any code of the method.

The paper fits parameters to velocities reconstructed from real videos of liquid
blobs and rivers (Sec. 3.3, Sec. 3.4.2, Sec. 4.4); those videos are not available,
so these recipes stand in for them:

* ``blurred_noise_mac``: N(0, 1) per MAC component drawn in C order (u, then v,
  then w), smoothed per component on its own staggered array by a separable
  Gaussian of sigma = 3 cells, radius 9, clamp-to-edge; wall-normal faces are
  then set to zero.
* ``ellipsoid_blob``: an ellipsoid resting on the floor (y = 0) with semi-axes
  a, c ~ U[0.40, 0.49] (in units of the box's y extent) and b set so that the
  ellipsoid fills 40 % of a unit box (clamped to <= 0.49); air elsewhere.
* ``sphere_union``: the union of 8 spheres with radii ~ U[20, 60] * n/256 cells
  and uniformly drawn centres, redrawn until the occupancy lies in [0.15, 0.50].
* ``random_mac``: unblurred N(0, 1) per MAC component (a strongly divergent
  right-hand side for the projection).
* ``gaussian_cloud``: Gaussians standing in for the generated and filled 3DGS
  assets (Sec. 3.3.1 fills the liquid with Gaussians at grid centres), one per
  liquid cell at a jittered position, covariance Q diag(s^2) Q^T with Q a random
  rotation and s ~ U[0.3, 0.9] dx per axis, opacity ~ U[0.3, 0.95] and
  degree-0 colour ~ U[0, 1]^3.
* ``look_at``: a pinhole camera on a sphere around a target (world y up), as
  (R, t, fx, fy, cx, cy) with x_c = R x + t and the vertical field of view given.

Array conventions (dense, C order, x fastest):
    cell arrays            shape (nz, ny, nx)
    u (x-velocity faces)   shape (nz, ny, nx + 1)
    v (y-velocity faces)   shape (nz, ny + 1, nx)
    w (z-velocity faces)   shape (nz + 1, ny, nx)
Cell types: 0 air, 1 liquid, 2 solid. Cells outside the array are solid walls.
"""
from __future__ import annotations

import numpy as np

AIR, LIQUID, SOLID = 0, 1, 2


def face_shapes(nx: int, ny: int, nz: int):
    """Dense shapes of the u, v, w face arrays."""
    return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)


def _blur_weights(sigma: float, radius: int) -> np.ndarray:
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    wts = np.exp(-0.5 * (x / sigma) ** 2)
    return wts / wts.sum()


def gaussian_blur3(a: np.ndarray, sigma: float = 3.0, radius: int = 9) -> np.ndarray:
    """Separable Gaussian blur with clamp-to-edge boundaries, float64."""
    from scipy.ndimage import correlate1d
    wts = _blur_weights(sigma, radius)
    out = np.asarray(a, dtype=np.float64)
    for axis in range(3):
        out = correlate1d(out, wts, axis=axis, mode="nearest")
    return out


def zero_wall_normal(u: np.ndarray, v: np.ndarray, w: np.ndarray) -> None:
    """Set the faces that lie on the box walls (normal velocity) to zero, in place."""
    u[:, :, 0] = 0.0
    u[:, :, -1] = 0.0
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    w[0, :, :] = 0.0
    w[-1, :, :] = 0.0


def random_mac(nx: int, ny: int, nz: int, seed: int, scale: float = 1.0):
    """Unblurred N(0, scale^2) MAC field, components drawn in C order u, v, w."""
    rng = np.random.default_rng(seed)
    return tuple(scale * rng.standard_normal(s) for s in face_shapes(nx, ny, nz))


def blurred_noise_mac(nx: int, ny: int, nz: int, seed: int, sigma_cells: float = 3.0,
                      radius: int = 9, scale: float = 1.0):
    """Seeded N(0,1) noise per component, Gaussian-blurred, wall-normal faces zeroed.

    The result is smooth but not divergence-free (the plain-forward workload)."""
    u, v, w = random_mac(nx, ny, nz, seed)
    u, v, w = (scale * gaussian_blur3(a, sigma_cells, radius) for a in (u, v, w))
    zero_wall_normal(u, v, w)
    return u, v, w


def all_liquid(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.full((nz, ny, nx), LIQUID, dtype=np.uint8)


def cell_centres(nx: int, ny: int, nz: int, dx: float):
    """World coordinates (x, y, z) of cell centres, each of shape (nz, ny, nx)."""
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                          (np.arange(nx) + 0.5) * dx, indexing="ij")
    return x, y, z


def ellipsoid_blob(nx: int, ny: int, nz: int, seed: int, occupancy: float = 0.40):
    """Liquid ellipsoid resting on the floor, air elsewhere; returns (types, info).

    Lengths are in units of the box's y extent (dx = 1/ny). The ellipsoid is
    centred over the middle of the floor at height b, so it touches y = 0."""
    rng = np.random.default_rng(seed)
    a, c = rng.uniform(0.40, 0.49, size=2)
    b = min(occupancy * 3.0 / (4.0 * np.pi * a * c), 0.49)
    dx = 1.0 / ny
    x, y, z = cell_centres(nx, ny, nz, dx)
    cx, cz = 0.5 * nx * dx, 0.5 * nz * dx
    inside = ((x - cx) / a) ** 2 + ((y - b) / b) ** 2 + ((z - cz) / c) ** 2 <= 1.0
    types = np.where(inside, LIQUID, AIR).astype(np.uint8)
    return types, {"a": float(a), "b": float(b), "c": float(c),
                   "occupancy": float(inside.mean())}


def sphere_union(nx: int, ny: int, nz: int, seed: int, count: int = 8,
                 occ_range=(0.15, 0.50), max_tries: int = 1000):
    """Union of `count` seeded spheres with radii U[20, 60] * n/256 cells; returns
    (types, info). Draws are repeated (same generator) until occupancy is in range."""
    rng = np.random.default_rng(seed)
    n = min(nx, ny, nz)
    k, j, i = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    for tries in range(1, max_tries + 1):
        radii = rng.uniform(20.0, 60.0, size=count) * n / 256.0
        centres = rng.uniform(0.0, 1.0, size=(count, 3)) * np.array([nx, ny, nz])
        inside = np.zeros((nz, ny, nx), dtype=bool)
        for r, (cx, cy, cz) in zip(radii, centres):
            inside |= (i - cx) ** 2 + (j - cy) ** 2 + (k - cz) ** 2 <= r * r
        occ = float(inside.mean())
        if occ_range[0] <= occ <= occ_range[1]:
            types = np.where(inside, LIQUID, AIR).astype(np.uint8)
            return types, {"occupancy": occ, "tries": tries}
    raise RuntimeError("sphere_union: no draw reached the occupancy range")


def river_with_blob(nx: int, ny: int, nz: int, seed: int, depth: float = 0.25):
    """Liquid blob on the floor plus a shallow liquid layer of the given depth (m);
    returns (types, inflow_u) where inflow_u flags the x = 0 wall faces of liquid
    cells below `depth` (dense u-face shape, uint8)."""
    types, info = ellipsoid_blob(nx, ny, nz, seed)
    dx = 1.0 / ny
    _, y, _ = cell_centres(nx, ny, nz, dx)
    types = np.where(y < depth, LIQUID, types).astype(np.uint8)
    inflow = np.zeros((nz, ny, nx + 1), dtype=np.uint8)
    inflow[:, :, 0] = (types[:, :, 0] == LIQUID) & (y[:, :, 0] < depth)
    info["occupancy"] = float((types == LIQUID).mean())
    return types, inflow, info


def weighted_band_target(nx: int, ny: int, nz: int, seed: int, scale: float = 1.0):
    """Independent smooth target field (seed offset by 100 from the initial field)."""
    return blurred_noise_mac(nx, ny, nz, seed + 100, scale=scale)


def gaussian_cloud(types: np.ndarray, dx: float, seed: int, jitter: float = 0.5):
    """(x (n, 3), opacity (n,), A (n, 3, 3), color (n, 3)) in float64, one Gaussian
    per liquid cell of `types` (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    k, j, i = np.nonzero(types == LIQUID)
    n = k.size
    x = (np.stack([i, j, k], axis=1) + 0.5 + jitter * (rng.random((n, 3)) - 0.5)) * dx
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, a, b, c = q.T
    Q = np.stack([1 - 2 * (b * b + c * c), 2 * (a * b - w * c), 2 * (a * c + w * b),
                  2 * (a * b + w * c), 1 - 2 * (a * a + c * c), 2 * (b * c - w * a),
                  2 * (a * c - w * b), 2 * (b * c + w * a), 1 - 2 * (a * a + b * b)], axis=1).reshape(n, 3, 3)
    sc = rng.uniform(0.3, 0.9, (n, 3)) * dx
    A = np.einsum("nij,nj,nkj->nik", Q, sc * sc, Q)
    opacity = rng.uniform(0.3, 0.95, n)
    color = rng.random((n, 3))
    return x, opacity, A, color


def look_at(target, radius: float, azimuth: float, elevation: float, width: int, height: int,
            fov_y: float = 0.8):
    """(R, t, fx, fy, cx, cy) of a camera at `radius` from `target`, looking at it;
    angles in radians, image y pointing down."""
    target = np.asarray(target, float)
    eye = target + radius * np.array([np.cos(elevation) * np.sin(azimuth), np.sin(elevation),
                                      np.cos(elevation) * np.cos(azimuth)])
    fwd = (target - eye) / np.linalg.norm(target - eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    f = 0.5 * height / np.tan(0.5 * fov_y)
    return R, t, f, f, 0.5 * width, 0.5 * height
