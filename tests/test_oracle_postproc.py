"""Pins of the oracle's post-processing (the figure quantities of Sect. 3):
current density j = curl B / mu0 and RK4 field lines along B/|B|.

The pins use facts that do not depend on the oracle's own code paths: the
tensor-product difference operators commute, so the discrete curl of a
discrete gradient vanishes to rounding; first differences are exact on
affine functions; trilinear interpolation reproduces affine fields, whose
field lines are straight lines or helices in closed form; classical RK4
converges at fourth order."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S


def _grid(pr):
    x = np.linspace(0.0, pr["Lx"], pr["nx"])
    y = np.linspace(0.0, pr["Ly"], pr["ny"])
    z = np.linspace(0.0, pr["Lz"], pr["nz"])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def test_curl_of_discrete_gradient_vanishes():
    """B = grad_h phi with numpy's second-order gradient (central inside,
    second-order one-sided at the ends: the field-recovery operators); the
    discrete curl of it is zero to rounding because differences along two
    different axes commute."""
    pr = S.problem(13, 11, 9, Lx=1.0, Ly=0.8, Lz=0.6, mu0=0.5)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((9, 11, 13))
    h = (pr["Lz"] / 8, pr["Ly"] / 10, pr["Lx"] / 12)
    gz, gy, gx = np.gradient(phi, *h, edge_order=2)
    J = oracle.current(pr, gx, gy, gz)
    scale = max(np.abs(g).max() for g in (gx, gy, gz)) / min(h)
    for k in ("jx", "jy", "jz"):
        assert np.abs(J[k]).max() < 1e-12 * scale, k
    # a non-gradient field does not give zero
    J2 = oracle.current(pr, gx, gz, gy)
    assert np.abs(J2["jmag"]).max() > 1e-3 * scale


def test_curl_of_affine_field_exact():
    """B = (c (z - y), c (x - z), c (y - x)) + const: curl B = (2c, 2c, 2c),
    exactly for the difference operators (exact on affine functions), so
    j = 2c/mu0 (1, 1, 1) at every node, faces included."""
    pr = S.problem(9, 7, 11, Lx=2.0, Ly=1.5, Lz=1.0, mu0=0.7)
    X, Y, Z = _grid(pr)
    c = 0.3
    Bx, By, Bz = c * (Z - Y) + 1.0, c * (X - Z) - 2.0, c * (Y - X) + 0.5
    J = oracle.current(pr, Bx, By, Bz)
    for k in ("jx", "jy", "jz"):
        assert np.allclose(J[k], 2 * c / 0.7, rtol=0, atol=1e-12)
    assert np.allclose(J["jmag"], 2 * c / 0.7 * math.sqrt(3), atol=1e-12)
    assert np.allclose(J["bmag"], np.sqrt(Bx ** 2 + By ** 2 + Bz ** 2), rtol=1e-15)


def test_straight_field_lines_of_uniform_field():
    pr = S.problem(9, 9, 9, Lx=1.0, Ly=1.0, Lz=1.0)
    shape = (9, 9, 9)
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    Bx, By, Bz = (np.full(shape, 5.0 * d[a]) for a in range(3))
    seeds = np.array([[0.1, 0.05, 0.0], [0.5, 0.503, 0.5], [1.2, 0.5, 0.5]])   # no exit exactly on a step
    ds = 0.01
    pts, lens = oracle.trace(pr, Bx, By, Bz, seeds, ds, 200)
    assert lens[2] == 0                                  # seed outside the box
    for q in range(2):
        # the line leaves through the face y = 1 or z = 1 (direction 2/3 in both)
        smax = min((1.0 - seeds[q, 1]) / d[1], (1.0 - seeds[q, 2]) / d[2])
        assert lens[q] == int(math.floor(smax / ds + 1e-9)) + 1
        s = ds * np.arange(lens[q])
        want = seeds[q][None, :] + s[:, None] * d[None, :]
        assert np.abs(pts[q, : lens[q]] - want).max() < 1e-13
    # backwards: against B
    pts_b, lens_b = oracle.trace(pr, Bx, By, Bz, seeds[1:2], ds, 200, direction=-1)
    s = ds * np.arange(lens_b[0])
    assert np.abs(pts_b[0, : lens_b[0]] - (seeds[1][None, :] - s[:, None] * d[None, :])).max() < 1e-13


def test_helical_field_lines_fourth_order():
    """B = (-(y - yc), x - xc, w) is affine, so trilinear interpolation is
    exact; its field lines are helices about (xc, yc).  At a fixed arc length
    the RK4 error falls by about 16 when ds halves."""
    pr = S.problem(17, 17, 17, Lx=2.0, Ly=2.0, Lz=4.0)
    X, Y, Z = _grid(pr)
    xc, yc, w = 1.0, 1.0, 0.8
    Bx, By, Bz = -(Y - yc), X - xc, np.full_like(X, w)
    R, th0 = 0.5, 0.3
    seed = np.array([[xc + R * math.cos(th0), yc + R * math.sin(th0), 0.2]])
    S_total = 3.0
    errs = []
    for ds in (0.1, 0.05, 0.025):
        n = int(round(S_total / ds))
        pts, lens = oracle.trace(pr, Bx, By, Bz, seed, ds, n)
        assert lens[0] == n + 1
        sp = math.sqrt(R * R + w * w)
        th = th0 + S_total / sp
        want = np.array([xc + R * math.cos(th), yc + R * math.sin(th), 0.2 + w * S_total / sp])
        errs.append(np.abs(pts[0, n] - want).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, errs


def test_field_line_stops_at_null():
    """|B| = 0 at the seed: the line is the seed alone."""
    pr = S.problem(5, 5, 5)
    X, Y, Z = _grid(pr)
    Bx, By, Bz = X - 0.5, Y - 0.5, -2 * (Z - 0.5)          # null at the centre (a node)
    pts, lens = oracle.trace(pr, Bx, By, Bz, np.array([[0.5, 0.5, 0.5]]), 0.01, 10)
    assert lens[0] == 1
