"""Pins of the oracle's qGGMRF prior (Sec. 3 Eqs. reg2, reg3; Sec. 5 hyper-parameters)."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(777)


def test_paper_hyper_parameters():
    with open(os.path.join(GOLDEN, "paper_prior_hyperparameters.json")) as fh:
        g = json.load(fh)
    assert oracle.PAPER_PRIOR["p"] == g["p"]
    assert abs(oracle.PAPER_PRIOR["sigma"] - 1.0 / g["sigma_inverse"]) < 1e-15
    assert oracle.PAPER_PRIOR["c"] == g["c"]


@pytest.mark.parametrize("dims,count", [(2, 8), (3, 26)])
def test_neighbourhood_and_weights(dims, count):
    offs, w = oracle.prior_weights(dims)
    assert len(offs) == count == len(set(offs))
    assert all(max(abs(v) for v in o) == 1 for o in offs)
    assert abs(w.sum() - 1.0) < 1e-15
    # inversely proportional to distance
    d = np.array([math.sqrt(sum(v * v for v in o)) for o in offs])
    assert np.allclose(w * d, (w * d)[0], rtol=1e-14)


def test_constant_image_has_zero_prior():
    f = np.full((3, 9, 9), 0.37)
    for dims in (2, 3):
        H, g = oracle.prior_value_grad(f, dims)
        assert H == 0.0 and np.abs(g).max() == 0.0


def test_two_pixel_closed_form():
    p, sigma, c = 1.2, 1.0 / 0.7, 1e-4
    a, b = 1.0, 0.0
    f = np.array([[[a, b]]])
    H, g = oracle.prior_value_grad(f, 2, p, sigma, c)
    # two ordered pairs, each with the axis weight 1/(4 + 4/sqrt 2)
    w1 = 1.0 / (4.0 + 4.0 / math.sqrt(2.0))
    u = abs(a - b) / sigma
    h = u ** 2 / (c + u ** (2 - p))
    assert abs(H - 2 * w1 * h) < 1e-15
    # the gradient is antisymmetric and matches the derivative of 2 w1 h
    assert abs(g[0, 0, 0] + g[0, 0, 1]) < 1e-15
    eps = 1e-6
    hp = (abs(a + eps - b) / sigma) ** 2 / (c + (abs(a + eps - b) / sigma) ** (2 - p))
    hm = (abs(a - eps - b) / sigma) ** 2 / (c + (abs(a - eps - b) / sigma) ** (2 - p))
    assert abs(g[0, 0, 0] - 2 * w1 * (hp - hm) / (2 * eps)) < 1e-8


def test_hand_value_at_unit_step():
    """Hand evaluation at f = [1, 0] with the paper's hyper-parameters:
    u = 0.7, u^0.8 = 0.7515..., h = 0.49/(1e-4 + u^0.8), H = 2 h / (4 + 2 sqrt 2)."""
    H, _ = oracle.prior_value_grad(np.array([[[1.0, 0.0]]]), 2)
    assert abs(H - 0.19088) < 5e-5


def test_corner_delta_border_rule():
    """Neighbours outside the image are left out; weights are not renormalised."""
    f = np.zeros((1, 5, 5))
    f[0, 0, 0] = 1.0
    H, _ = oracle.prior_value_grad(f, 2)
    _, w = oracle.prior_weights(2)
    w1, w2 = w.max(), w.min()
    h = oracle.rho(1.0, 1.2, 1.0 / 0.7, 1e-4)
    # the corner has 2 axis and 1 diagonal neighbour; each pair counted twice
    assert abs(H - 2 * (2 * w1 + w2) * h) < 1e-14


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("scale", [1e-5, 1e-2, 1.0])
def test_gradient_matches_central_differences(dims, scale):
    f = scale * RNG.standard_normal((3, 6, 6))
    _, g = oracle.prior_value_grad(f, dims)
    for _ in range(6):
        d = RNG.standard_normal(f.shape)
        h = 1e-6 * scale
        Hp, _ = oracle.prior_value_grad(f + h * d, dims)
        Hm, _ = oracle.prior_value_grad(f - h * d, dims)
        fd = (Hp - Hm) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12) + 1e-9, (fd, an)


def test_rho_prime_matches_difference_quotient():
    p, s, c = 1.2, 1.0 / 0.7, 1e-4
    for dlt in (-2.0, -1e-3, 1e-6, 0.3, 5.0):
        e = 1e-7 * max(abs(dlt), 1e-6)
        fd = (oracle.rho(dlt + e, p, s, c) - oracle.rho(dlt - e, p, s, c)) / (2 * e)
        assert abs(fd - oracle.rho_prime(dlt, p, s, c)) <= 1e-5 * abs(fd) + 1e-12


def test_lipschitz_bound_dominates_curvature():
    p, s, c = 1.2, 1.0 / 0.7, 1e-4
    L = oracle.prior_lipschitz(p, s, c)
    # Rayleigh quotients of the Hessian (by differences of the gradient)
    f = 1e-3 * RNG.standard_normal((2, 8, 8))
    for dims in (2, 3):
        _, g0 = oracle.prior_value_grad(f, dims, p, s, c)
        for _ in range(5):
            d = RNG.standard_normal(f.shape)
            d /= np.linalg.norm(d)
            _, g1 = oracle.prior_value_grad(f + 1e-7 * d, dims, p, s, c)
            q = float(np.sum((g1 - g0) * d)) / 1e-7
            assert q <= L * (1 + 1e-6)
