"""Pins of the FP64 oracle's Radon operator A and adjoint A^T.

Each test fixes the oracle to something other than itself:
  * analytic projections of a Gaussian (continuous Radon transform,
    Sec. 2.1 Eq. radon_transform; band-limited so the discrete operator must
    reproduce it to rounding) -- pins scale, centre, sign of theta, direction
    of t and the detector origin;
  * theta = 0 and theta = pi/2, where the operator must reduce exactly to
    column and row sums;
  * mass conservation (sum over bins equals the image sum at every angle);
  * an 8x8 system matrix built entry by entry from the Dirichlet closed form
    (a different formula from the oracle's two-stage NUDFT);
  * the adjoint identity <Ax, y> = <x, A^T y>;
  * analytic ellipse line integrals (coarse: pixelisation error).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_12934_gb300 import synth

RNG = np.random.default_rng(12345)


def test_dirichlet_kernel_special_values():
    for D in (12, 92, 184):
        assert oracle.dirichlet(D, 0.0) == 1.0
        for k in (1, 2, 5, D - 1, D + 3, -7):
            if k % D:
                assert abs(oracle.dirichlet(D, float(k))) < 1e-13
        # D-periodic
        u = 3.37
        assert abs(oracle.dirichlet(D, u) - oracle.dirichlet(D, u + D)) < 1e-12
        # mean value over one period of unit-spaced samples is 1/D * D = 1
        s = sum(oracle.dirichlet(D, i - D / 2 - 0.318) for i in range(D))
        assert abs(s - 1.0) < 1e-12


@pytest.mark.parametrize("cx,cy,s", [(5.3, -7.1, 3.0), (-9.0, 2.5, 2.9), (0.0, 0.0, 3.6)])
def test_gaussian_blob_matches_analytic_projection(cx, cy, s):
    N, A, D = 64, 12, 92
    th = np.sort(RNG.uniform(0.0, math.pi, A))
    f = synth.gaussian_blob(N, cx, cy, s)
    y = oracle.radon_fwd(f, A, D, th)
    ya = synth.gaussian_line_integrals(cx, cy, s, th, D)
    assert np.abs(y - ya).max() <= 1e-10 * np.abs(ya).max()


def test_theta_zero_and_half_pi_are_column_and_row_sums():
    N, D = 32, 52
    x = RNG.standard_normal((N, N))
    y = oracle.radon_fwd(x, 2, D, np.array([0.0, math.pi / 2]))
    off = (D - N) // 2
    col = x.sum(axis=0)  # sum over iy for every ix
    row = x.sum(axis=1)  # sum over ix for every iy
    assert np.abs(y[0, off:off + N] - col).max() < 1e-11
    assert np.abs(y[1, off:off + N] - row).max() < 1e-11
    assert np.abs(y[0, :off]).max() < 1e-11 and np.abs(y[0, off + N:]).max() < 1e-11


def test_mass_conservation_every_angle():
    N, A, D = 40, 9, 60
    x = RNG.standard_normal((N, N))
    th = RNG.uniform(0.0, math.pi, A)
    y = oracle.radon_fwd(x, A, D, th)
    assert np.abs(y.sum(axis=1) - x.sum()).max() < 1e-10


def _closed_form_matrix(N, D, th):
    """System matrix M[(a,i), (iy,ix)] = K_D(t_i - s_n(a)), written out."""
    c = np.arange(N) - N // 2
    X, Y = np.meshgrid(c, c)
    rows = []
    for a in range(th.shape[0]):
        s = (X * math.cos(th[a]) + Y * math.sin(th[a])).ravel()
        for i in range(D):
            u = (i - D // 2) - s
            r = np.mod(u + D / 2, D) - D / 2
            with np.errstate(invalid="ignore", divide="ignore"):
                k = (np.sin(math.pi * r * (D - 1) / D) / np.sin(math.pi * r / D)
                     + np.cos(math.pi * r)) / D
            k[r == 0.0] = 1.0
            rows.append(k)
    return np.array(rows)


def test_dense_8x8_system_matrix_and_transpose():
    N, A, D = 8, 5, 12
    th = RNG.uniform(0.0, math.pi, A)
    M = _closed_form_matrix(N, D, th)
    E = np.eye(N * N).reshape(N * N, N, N)
    cols = oracle.radon_fwd(E, A, D, th).reshape(N * N, A * D).T
    assert np.abs(cols - M).max() < 1e-12
    Ey = np.eye(A * D).reshape(A * D, A, D)
    rows = oracle.radon_adj(Ey, N, th).reshape(A * D, N * N)
    assert np.abs(rows - M).max() < 1e-12


def test_adjoint_identity_random():
    N, A, D = 48, 17, 70
    th = RNG.uniform(0.0, math.pi, A)
    x = RNG.standard_normal((N, N))
    y = RNG.standard_normal((A, D))
    lhs = float(np.sum(oracle.radon_fwd(x, A, D, th) * y))
    rhs = float(np.sum(x * oracle.radon_adj(y, N, th)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_sampled_entries_agree_with_full_operator():
    N, A, D = 32, 11, 46
    th = RNG.uniform(0.0, math.pi, A)
    x = RNG.standard_normal((N, N))
    y = RNG.standard_normal((A, D))
    ai = RNG.integers(0, A, 30)
    ii = RNG.integers(0, D, 30)
    full = oracle.radon_fwd(x, A, D, th)
    assert np.abs(oracle.radon_fwd_at(x, A, D, ai, ii, th) - full[ai, ii]).max() < 1e-11
    pix = RNG.integers(0, N * N, 30)
    fullx = oracle.radon_adj(y, N, th).ravel()
    assert np.abs(oracle.radon_adj_at(y, N, pix, th) - fullx[pix]).max() < 1e-11


def test_batch_is_slice_by_slice():
    N, A, D = 16, 6, 24
    x = RNG.standard_normal((3, N, N))
    yb = oracle.radon_fwd(x, A, D)
    for k in range(3):
        assert np.array_equal(yb[k], oracle.radon_fwd(x[k], A, D))


def test_ellipse_phantom_close_to_analytic_line_integrals():
    N, A, D = 128, 30, synth.det_for(128)
    ells = synth.random_ellipses(N, synth.BASE_SEED)
    f = synth.rasterize(N, ells)
    th = oracle.default_angles(A)
    y = oracle.radon_fwd(f, A, D, th)
    ya = synth.ellipse_line_integrals(ells, th, D)
    rel = np.linalg.norm(y - ya) / np.linalg.norm(ya)
    assert rel < 0.05, rel


def test_rejects_odd_detector_width():
    with pytest.raises(ValueError):
        oracle.radon_fwd(np.zeros((8, 8)), 4, 11)


@pytest.mark.parametrize("delta", [2.7, -5.25, 0.5])
def test_rotation_axis_offset_moves_the_gaussian_projection(delta):
    """With the axis at detector coordinate D/2 + delta, the projection of a
    Gaussian is the analytic one shifted by +delta along t (Sec. 4.1)."""
    N, A, D = 64, 10, 92
    th = np.sort(RNG.uniform(0.0, math.pi, A))
    cx, cy, s = 4.1, -6.3, 3.0
    f = synth.gaussian_blob(N, cx, cy, s)
    y = oracle.radon_fwd(f, A, D, th, delta=delta)
    t = np.arange(D) - D // 2
    tc = cx * np.cos(th) + cy * np.sin(th) + delta
    ya = math.sqrt(2 * math.pi) * s * np.exp(-(t[None, :] - tc[:, None]) ** 2 / (2 * s * s))
    assert np.abs(y - ya).max() <= 1e-10 * np.abs(ya).max()


def test_shifted_operator_adjoint_and_sampled_forms():
    N, A, D, delta = 32, 9, 46, 1.37
    th = RNG.uniform(0.0, math.pi, A)
    x = RNG.standard_normal((N, N))
    y = RNG.standard_normal((A, D))
    Ax = oracle.radon_fwd(x, A, D, th, delta=delta)
    Aty = oracle.radon_adj(y, N, th, delta=delta)
    assert abs(float(np.sum(Ax * y)) - float(np.sum(x * Aty))) <= 1e-11 * abs(float(np.sum(Ax * y)))
    ai = RNG.integers(0, A, 20)
    ii = RNG.integers(0, D, 20)
    assert np.abs(oracle.radon_fwd_at(x, A, D, ai, ii, th, delta=delta) - Ax[ai, ii]).max() < 1e-11
    pix = RNG.integers(0, N * N, 20)
    assert np.abs(oracle.radon_adj_at(y, N, pix, th, delta=delta) - Aty.ravel()[pix]).max() < 1e-11
    # an integer offset at theta = 0 shifts the column sums by exactly delta bins
    y0 = oracle.radon_fwd(x, 1, D, np.array([0.0]), delta=3.0)[0]
    off = (D - N) // 2 + 3
    assert np.abs(y0[off:off + N] - x.sum(axis=0)).max() < 1e-11
