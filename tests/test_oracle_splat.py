"""Pins of the oracle's FP32 projection + count splat (Appendix A render pipeline).

Brute-force closed forms on tiny inputs: pixel-centre grids give an all-ones
image; window edges (lower edge kept, upper edge dropped), non-finite and
out-of-window values are dropped; the 3D path with an identity matrix reduces
to the 2D window [-1,1)^2; points behind the camera are dropped; a point on the
camera axis lands on the centre pixel.
"""
import numpy as np
import pytest

import oracle
from paper_1505_00344_gb300.workloads import look_at_perspective, random_states


@pytest.mark.parametrize("W,H", [(1, 1), (7, 5), (64, 48)])
def test_pixel_centres_fill_image_once(W, H):
    lo, hi = (-3.0, 10.0), (5.0, 20.0)
    c, r = np.meshgrid(np.arange(W), np.arange(H))
    u = lo[0] + (c.ravel() + 0.5) * (hi[0] - lo[0]) / W
    v = lo[1] + (r.ravel() + 0.5) * (hi[1] - lo[1]) / H
    img = oracle.splat2d(u, v, lo, hi, W, H)
    assert img.dtype == np.uint32 and img.shape == (H, W)
    assert (img == 1).all()


def test_edges_and_specials():
    W, H = 10, 4
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    u = np.array([0.0, 0.99999994, 1.0, -1e-7, np.nan, np.inf, -np.inf, 0.5, 0.5, 3e38],
                 dtype=np.float32)
    v = np.array([0.0, 0.99999994, 0.5, 0.5, 0.5, 0.5, 0.5, np.nan, 1.0, 0.5], dtype=np.float32)
    img = oracle.splat2d(u, v, lo, hi, W, H)
    assert img[0, 0] == 1  # lower edges kept
    assert img[H - 1, W - 1] == 1  # just below upper edges
    assert img.sum() == 2  # everything else dropped


def test_rows_are_bottom_up_and_counts_add():
    W, H = 4, 4
    u = np.full(5, 0.1, dtype=np.float32)
    v = np.array([0.1, 0.1, 0.9, 0.9, 0.9], dtype=np.float32)
    img = oracle.splat2d(u, v, (0, 0), (1, 1), W, H)
    assert img[0, 0] == 2 and img[3, 0] == 3 and img.sum() == 5
    img2 = oracle.splat2d(u, v, (0, 0), (1, 1), W, H, image=img)  # accumulate
    assert img2[3, 0] == 6


def test_include_mask():
    u = np.array([0.1, 0.2, 0.3], dtype=np.float32)
    v = np.array([0.5, 0.5, 0.5], dtype=np.float32)
    img = oracle.splat2d(u, v, (0, 0), (1, 1), 10, 1, include=np.array([1, 0, 1], np.uint8))
    assert img[0].tolist() == [0, 1, 0, 1, 0, 0, 0, 0, 0, 0]


def test_identity_3d_reduces_to_2d():
    # non-finite x or y are dropped by both paths; a non-finite z would poison the 3D
    # product (0 * inf) so z stays finite here
    x = random_states(3, 5000, [-1.2, -1.2, -5], [1.2, 1.2, 5], seed=3, specials=True)
    x[2] = random_states(1, 5000, [-5], [5], seed=4)[0]
    eye = np.eye(4, dtype=np.float32).T.reshape(16)
    a = oracle.splat3d(x[0], x[1], x[2], eye, 33, 17)
    b = oracle.splat2d(x[0], x[1], (-1.0, -1.0), (1.0, 1.0), 33, 17)
    np.testing.assert_array_equal(a, b)


def test_behind_camera_dropped_and_axis_hits_centre():
    W, H = 64, 32
    mvp = look_at_perspective((0.0, 0.0, 10.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, W / H,
                              0.1, 100.0)
    # points along the view axis, in front of the camera -> centre pixel (W/2, H/2)
    z = np.array([5.0, 0.0, -20.0], dtype=np.float32)
    img = oracle.splat3d(np.zeros(3, np.float32), np.zeros(3, np.float32), z, mvp, W, H)
    assert img[H // 2, W // 2] == 3 and img.sum() == 3
    # behind the camera (z > 10): clip w < 0 -> dropped
    img = oracle.splat3d(np.array([0.0, 1.0], np.float32), np.zeros(2, np.float32),
                         np.array([11.0, 50.0], np.float32), mvp, W, H)
    assert img.sum() == 0
    # symmetric points land in mirrored columns
    img = oracle.splat3d(np.array([-1.0, 1.0], np.float32), np.zeros(2, np.float32),
                         np.zeros(2, np.float32), mvp, W, H)
    cols = np.nonzero(img.sum(axis=0))[0]
    assert len(cols) == 2 and cols[0] + cols[1] == W - 1


def test_count_conservation_random():
    x = random_states(2, 20000, [-1, -1], [2, 2], seed=9, specials=True)
    img = oracle.splat2d(x[0], x[1], (0.0, 0.0), (1.0, 1.0), 50, 40)
    inside = ((x[0] >= 0) & (x[0] < 1) & (x[1] >= 0) & (x[1] < 1)).sum()
    # values within one float ulp of the upper edge could round into the window; the sample
    # has none there, so the counts agree exactly
    assert img.sum() == inside


def test_general_matrix_maps_points_to_pixel_centres():
    # rows of M (column-major storage m[4*col + row]):
    #   clip.x = 0.5 y + 0.1,  clip.y = 2 x - 0.3,  clip.z = z,  clip.w = 0.5 z + 1
    # points with z = 2 (w = 2) chosen so that clip.xy / w hits every pixel centre once
    W, H = 24, 10
    M = np.array([[0.0, 0.5, 0.0, 0.1],
                  [2.0, 0.0, 0.0, -0.3],
                  [0.0, 0.0, 1.0, 0.0],
                  [0.0, 0.0, 0.5, 1.0]])
    m = M.T.reshape(16).astype(np.float32)
    c, r = np.meshgrid(np.arange(W), np.arange(H))
    nx = -1.0 + (c.ravel() + 0.5) * 2.0 / W
    ny = -1.0 + (r.ravel() + 0.5) * 2.0 / H
    y = (2.0 * nx - 0.1) / 0.5
    x = (2.0 * ny + 0.3) / 2.0
    z = np.full_like(x, 2.0)
    img = oracle.splat3d(x, y, z, m, W, H)
    assert (img == 1).all()
