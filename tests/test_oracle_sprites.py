"""Pins of the oracle's soft-sprite render technique (Appendix A: a square on the
screen centred on each projected particle, an intensity falling off with the
distance from the centre, GL_SRC_ALPHA / GL_ONE additive blending into colour
channels).

Reading pinned here: pixel centres at (col + 1/2, row + 1/2); half-side R; q = d^2/R^2;
intensity (1 - q)^2 for q < 1; channel k gains gain * intensity * colour[group][k].

* a hand-computed case (dyadic numbers, so every value is exact);
* the closed form of the sprite's mass: the continuous integral of (1 - r^2/R^2)^2 over
  the disc is pi R^2 / 3, which the pixel-lattice sum approaches as R grows;
* exact mirror and transpose symmetry about a pixel centre;
* translation: a sprite cut by the window edge equals the crop of an uncut one;
* groups and colours: the image is the sum over groups of colour x density;
* the 3D path reduces to the 2D one under an orthographic matrix, and the footprint
  on screen does not depend on depth;
* particles that are behind the camera or not finite draw nothing.
"""
import numpy as np

import oracle

ONE = [1.0, 0.0, 0.0, 0.0]


def window(W, H):
    return [0.0, 0.0], [float(W), float(H)]  # scale 1: state coordinates are pixel coordinates


def test_hand_computed_two_pixels():
    lo, hi = window(64, 64)
    img, aimg, frags = oracle.sprites2d([10.25], [20.5], lo, hi, 64, 64, 1.0, 2.0, [1.0, 2.0, 0.5, -1.0])
    # centre (10.25, 20.5): pixel (10, 20) has dx = 0.25, q = 1/16, a = (15/16)^2;
    # pixel (9, 20) has dx = -0.75, q = 9/16, a = (7/16)^2; every other centre is >= 1 away
    a10, a9 = (15 / 16) ** 2, (7 / 16) ** 2
    want = np.zeros((64, 64, 4))
    want[20, 10] = 2.0 * a10 * np.array([1.0, 2.0, 0.5, -1.0])
    want[20, 9] = 2.0 * a9 * np.array([1.0, 2.0, 0.5, -1.0])
    np.testing.assert_array_equal(img, want)
    np.testing.assert_array_equal(aimg, np.abs(want))
    assert frags.sum() == 2 and frags[20, 10] == 1 and frags[20, 9] == 1


def test_rim_is_excluded():
    # at a pixel centre with R = 1 the four neighbours sit exactly on the rim (q = 1)
    lo, hi = window(16, 16)
    img, _, frags = oracle.sprites2d([5.5], [7.5], lo, hi, 16, 16, 1.0, 1.0, ONE)
    assert frags.sum() == 1 and img[7, 5, 0] == 1.0 and img[:, :, 0].sum() == 1.0


def test_mass_approaches_closed_form():
    W = 101
    lo, hi = window(W, W)
    for R, centre, tol in [(8.0, (50.5, 50.5), 2e-4), (24.0, (50.5, 50.5), 1e-5), (8.0, (50.3, 50.8), 2e-4),
                           (24.0, (49.9, 50.15), 1e-5)]:
        img, _, _ = oracle.sprites2d([centre[0]], [centre[1]], lo, hi, W, W, R, 1.0, ONE)
        mass = img[:, :, 0].sum()
        assert abs(mass / (np.pi * R * R / 3.0) - 1.0) <= tol, (R, centre, mass)


def test_symmetric_about_a_pixel_centre():
    lo, hi = window(33, 33)
    img, _, _ = oracle.sprites2d([16.5], [16.5], lo, hi, 33, 33, 5.5, 1.0, ONE)
    d = img[:, :, 0]
    np.testing.assert_array_equal(d, d[::-1, :])
    np.testing.assert_array_equal(d, d[:, ::-1])
    np.testing.assert_array_equal(d, d.T)
    # row 0 is the bottom of the window: a particle low in v lands in low rows
    img, _, _ = oracle.sprites2d([16.5], [3.5], lo, hi, 33, 33, 2.0, 1.0, ONE)
    rows = np.nonzero(img[:, :, 0].sum(axis=1))[0]
    assert rows.min() == 2 and rows.max() == 4


def test_window_edge_cuts_the_sprite():
    # a sprite centred 1.25 px left of the window, seen in a window padded by 8 px
    R = 3.0
    cut, _, _ = oracle.sprites2d([-1.25], [10.5], [0.0, 0.0], [32.0, 32.0], 32, 32, R, 1.0, ONE)
    full, _, _ = oracle.sprites2d([-1.25], [10.5], [-8.0, -8.0], [40.0, 40.0], 48, 48, R, 1.0, ONE)
    np.testing.assert_array_equal(cut, full[8:40, 8:40])
    assert cut[:, :, 0].sum() > 0 and full[:, :, 0].sum() > cut[:, :, 0].sum()


def test_groups_and_colours_are_linear():
    rng = np.random.default_rng(3)
    W, H = 40, 30
    lo, hi = window(W, H)
    u = rng.uniform(-2, W + 2, 300).astype(np.float32)
    v = rng.uniform(-2, H + 2, 300).astype(np.float32)
    g = rng.integers(0, 3, 300).astype(np.int32)
    colours = np.array([[1.0, 0.2, 0.0, 0.5], [0.0, 1.0, 0.3, -0.5], [0.25, 0.25, 1.0, 2.0]])
    img, _, _ = oracle.sprites2d(u, v, lo, hi, W, H, 2.5, 0.7, colours, group=g)
    want = np.zeros((H, W, 4))
    for k in range(3):
        dens, _, _ = oracle.sprites2d(u, v, lo, hi, W, H, 2.5, 1.0, ONE, include=(g == k))
        want += 0.7 * dens[:, :, :1] * colours[k][None, None, :]
    np.testing.assert_allclose(img, want, rtol=1e-12, atol=1e-12)


def test_3d_orthographic_matches_2d_and_depth_does_not_scale():
    W, H = 64, 32
    # column-major: x_ndc = x * 2/W - 1, y_ndc = y * 2/H - 1, w = 1 (all dyadic, so exact)
    m = np.zeros(16, np.float32)
    m[0], m[5], m[10], m[15] = 2.0 / W, 2.0 / H, 1.0, 1.0
    m[12], m[13] = -1.0, -1.0
    xs = np.array([10.25, 40.5, 3.75, 63.0], np.float32)
    ys = np.array([20.5, 5.25, 31.0, 16.0], np.float32)
    zs = np.array([0.0, 5.0, -3.0, 1.0], np.float32)
    i3, _, f3 = oracle.sprites3d(xs, ys, zs, m, W, H, 2.5, 1.0, ONE)
    i2, _, f2 = oracle.sprites2d(xs, ys, [0.0, 0.0], [float(W), float(H)], W, H, 2.5, 1.0, ONE)
    np.testing.assert_array_equal(i3, i2)
    np.testing.assert_array_equal(f3, f2)
    # perspective: w = z, so (x, y, z) and (2x, 2y, 2z) project to one point; same footprint
    p = np.zeros(16, np.float32)
    p[0], p[5], p[11] = 1.0, 1.0, 1.0  # clip = (x, y, 0, z)
    a, _, _ = oracle.sprites3d([0.25], [-0.5], [1.0], p, W, H, 3.0, 1.0, ONE)
    b, _, _ = oracle.sprites3d([0.5], [-1.0], [2.0], p, W, H, 3.0, 1.0, ONE)
    np.testing.assert_array_equal(a, b)
    assert a[:, :, 0].sum() > 0
    # behind the camera (w <= 0) and non-finite particles draw nothing
    c, _, _ = oracle.sprites3d([0.25, np.nan, np.inf], [-0.5, 0.0, 0.0], [-1.0, 1.0, 1.0], p, W, H, 3.0, 1.0, ONE)
    assert not c.any()
    d, _, _ = oracle.sprites2d([np.nan, np.inf, -np.inf, 1e30], [1.0, 1.0, 1.0, 1.0], [0.0, 0.0], [8.0, 8.0],
                               8, 8, 2.0, 1.0, ONE)
    assert not d.any()
