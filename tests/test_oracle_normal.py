"""Pins of the oracle's normal operator A^T A (the Hessian of the unweighted data
term, Sec. 3 Eqs. gradient and transpose), and of the reading of the discrete
operator that the GPU normal operator is built on.

For the discrete operator (even D, the Nyquist pair m = +-D/2 weighted 1/2,
rotation-axis offset delta), the sum over the detector bins t_i = i - D/2 of
two shifted Dirichlet kernels K has a closed form:

    sum_i K(t_i - u) K(t_i - v) = K(u - v) - cos(pi (u - v)) / 2D
                                           + cos(pi (u + v)) / 2D,

so A^T A is Toeplitz plus Hankel in the centred pixel coordinates p:

    (A^T A f)(p') = sum_p f(p) [T(p' - p) + H(p' + p)],
    T(d) = sum_a K(s_d(a)) - cos(pi s_d(a)) / 2D,
    H(e) = sum_a cos(pi (s_e(a) + 2 delta)) / 2D,
    s_d(a) = d_x cos(theta_a) + d_y sin(theta_a).

Both terms are 2N-periodic convolutions after embedding (|d| < N, -N <= e < N),
so A^T A f = IDFT(T^ F(k) + H^ F(-k)) on the 2N x 2N grid.

The tests check the oracle (a composition of the exact NUDFT operators)
against brute-force sums built here from the closed form of K alone, and check
the embedding with numpy's FFT.  A dropped Nyquist term, a wrong sign of
delta, or a transposed index fails one of them.
"""
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20230426)


def kdir(D, u):
    """K_D(u) = (1/D) [sin(pi u (D-1)/D) / sin(pi u / D) + cos(pi u)], K_D(0) = 1
    (even D; D-periodic)."""
    u = np.asarray(u, np.float64)
    r = u - D * np.rint(u / D)
    den = np.sin(np.pi * r / D)
    with np.errstate(invalid="ignore", divide="ignore"):
        k = (np.sin(np.pi * r * (D - 1) / D) / den + np.cos(np.pi * u)) / D
    return np.where(r == 0.0, 1.0, k)


def tk_terms(D, s, delta):
    """Per-angle Toeplitz and Hankel terms at projection coordinate s."""
    t = kdir(D, s) - np.cos(np.pi * s) / (2 * D)
    h = np.cos(np.pi * (s + 2.0 * delta)) / (2 * D)
    return t, h


def brute_normal(f, theta, D, delta):
    N = f.shape[0]
    c = np.arange(N) - N // 2
    py, px = np.meshgrid(c, c, indexing="ij")
    px, py = px.ravel().astype(np.float64), py.ravel().astype(np.float64)
    fv = f.ravel()
    out = np.zeros(N * N)
    for th in theta:
        s = px * math.cos(th) + py * math.sin(th)          # s_p(a) for every pixel
        sd = s[:, None] - s[None, :]                          # s_{p' - p}
        se = s[:, None] + s[None, :]                          # s_{p' + p}
        t, _ = tk_terms(D, sd, delta)
        _, h = tk_terms(D, se, delta)
        out += (t + h) @ fv
    return out.reshape(N, N)


def embedded_normal(f, theta, D, delta):
    """A^T A f through the 2N-periodic embedding, with numpy's FFT."""
    N = f.shape[0]
    G = 2 * N
    j = np.arange(G)
    d = np.where(j < N, j, j - G).astype(np.float64)    # index j <-> coordinate d (mod G)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    T = np.zeros((G, G))
    H = np.zeros((G, G))
    for th in theta:
        s = dx * math.cos(th) + dy * math.sin(th)
        t, h = tk_terms(D, s, delta)
        T += t
        H += h
    fe = np.zeros((G, G))
    c = (np.arange(N) - N // 2) % G
    fe[np.ix_(c, c)] = f
    F = np.fft.fft2(fe)
    Fm = F[(-j) % G][:, (-j) % G]                         # F(-k)
    out = np.fft.ifft2(np.fft.fft2(T) * F + np.fft.fft2(H) * Fm)
    return out[np.ix_(c, c)], np.fft.fft2(T)


@pytest.mark.parametrize("D", [12, 14, 40])
def test_bin_sum_closed_form(D):
    t = np.arange(D) - D / 2
    for _ in range(20):
        u, v = RNG.uniform(-2 * D, 2 * D, 2)
        lhs = float(np.sum(kdir(D, t - u) * kdir(D, t - v)))
        rhs = (float(kdir(D, u - v)) - math.cos(math.pi * (u - v)) / (2 * D)
               + math.cos(math.pi * (u + v)) / (2 * D))
        assert abs(lhs - rhs) < 1e-12
    # the Hankel term is really there: without it the identity fails
    u, v = 0.3, 1.1
    lhs = float(np.sum(kdir(D, t - u) * kdir(D, t - v)))
    assert abs(lhs - (float(kdir(D, u - v)) - math.cos(math.pi * (u - v)) / (2 * D))) > 1e-4


@pytest.mark.parametrize("delta", [0.0, 0.37, -1.25])
@pytest.mark.parametrize("theta", ["default", "wide"])
def test_oracle_normal_matches_toeplitz_plus_hankel(delta, theta):
    N, A, D = 8, 5, 12
    th = oracle.default_angles(A) if theta == "default" else np.array([0.1, 1.3, 2.9, 3.7, -0.8])
    f = RNG.standard_normal((N, N))
    got = oracle.normal_op(f, A, D, th, delta)
    ref = brute_normal(f, th, D, delta)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("delta", [0.0, 0.6])
def test_embedding_reproduces_normal(delta):
    N, A, D = 8, 7, 14
    th = oracle.default_angles(A)
    f = RNG.standard_normal((N, N))
    out, That = embedded_normal(f, th, D, delta)
    ref = oracle.normal_op(f, A, D, th, delta)
    assert np.max(np.abs(out.imag)) < 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(out.real - ref)) < 1e-11 * np.max(np.abs(ref))
    # T is even, so its spectrum is real
    assert np.max(np.abs(That.imag)) < 1e-10 * np.max(np.abs(That.real))


def test_normal_quadratic_form_is_projection_energy():
    N, A, D = 16, 9, 24
    f = RNG.standard_normal((2, N, N))
    g = RNG.standard_normal((2, N, N))
    nf = oracle.normal_op(f, A, D)
    ng = oracle.normal_op(g, A, D)
    yf = oracle.radon_fwd(f, A, D)
    assert abs(np.sum(f * nf) - np.sum(yf * yf)) < 1e-10 * np.sum(yf * yf)
    assert abs(np.sum(g * nf) - np.sum(f * ng)) < 1e-10 * np.sum(yf * yf)
    # slices are independent
    assert np.allclose(oracle.normal_op(f[1], A, D), nf[1], rtol=0, atol=1e-12 * np.abs(nf).max())
