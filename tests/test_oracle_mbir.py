"""Pins of the oracle's MBIR pieces (Sec. 3: objective, gradient, optimizer).

The optimizer's iterates are not printed in the paper; these tests pin what
mathematics fixes: the gradient of the objective (central differences), the
power-iteration norm (dense eigenvalue), and that with no prior and unit
weights the accelerated gradient with restart converges to the least-squares
solution of the dense system (normal equations).
"""
import math

import numpy as np

import oracle
from test_oracle_radon import _closed_form_matrix

RNG = np.random.default_rng(4242)


def _tiny(N=8, A=24, D=14):
    th = oracle.default_angles(A)
    return th, _closed_form_matrix(N, D, th)


def test_data_gradient_is_dense_normal_equation_residual():
    N, A, D = 8, 10, 14
    th, M = _tiny(N, A, D)
    x = RNG.standard_normal((1, N, N))
    b = RNG.standard_normal((1, A, D))
    w = RNG.uniform(0.2, 1.0, (1, A, D))
    G, g = oracle.data_grad(x, b, w, th)
    r = M @ x.ravel() - b.ravel()
    assert abs(G - 0.5 * np.sum(w.ravel() * r * r)) < 1e-10
    assert np.abs(g.ravel() - M.T @ (w.ravel() * r)).max() < 1e-10


def test_objective_gradient_matches_central_differences():
    N, A, D = 8, 12, 14
    th = oracle.default_angles(A)
    x = 0.3 * RNG.standard_normal((2, N, N))
    b = RNG.standard_normal((2, A, D))
    w = RNG.uniform(0.2, 1.0, (2, A, D))
    lam = 0.05
    prior = oracle.PAPER_PRIOR
    G, H, g = oracle.objective_grad(x, b, w, lam, prior, 3, th)
    for _ in range(4):
        d = RNG.standard_normal(x.shape)
        h = 1e-6
        Gp, Hp, _ = oracle.objective_grad(x + h * d, b, w, lam, prior, 3, th)
        Gm, Hm, _ = oracle.objective_grad(x - h * d, b, w, lam, prior, 3, th)
        fd = ((Gp + Hp) - (Gm + Hm)) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7


def test_power_norm_matches_dense_eigenvalue():
    N, A, D = 8, 10, 14
    th, M = _tiny(N, A, D)
    w = RNG.uniform(0.2, 1.0, (1, A, D))
    lam = oracle.power_norm(N, A, D, w, RNG.standard_normal((1, N, N)), 300, th)
    ev = np.linalg.eigvalsh(M.T @ (w.ravel()[:, None] * M)).max()
    assert abs(lam - ev) <= 1e-8 * ev


def test_no_prior_unit_weight_converges_to_least_squares():
    N, A, D = 8, 24, 14
    th, M = _tiny(N, A, D)
    xt = RNG.standard_normal((N, N))
    b = (M @ xt.ravel()).reshape(1, A, D) + 0.01 * RNG.standard_normal((1, A, D))
    xls = np.linalg.lstsq(M, b.ravel(), rcond=None)[0]
    L = np.linalg.norm(M, 2) ** 2
    x, log = oracle.mbir_solve(b, None, N, 4000, 1.0 / L, lam=0.0, theta=th, return_log=True)
    assert np.linalg.norm(x.ravel() - xls) <= 1e-8 * np.linalg.norm(xls)
    assert any(e["restart"] for e in log)
    # the same schedule without restart is markedly slower on this problem
    x_nr = oracle.mbir_solve(b, None, N, 4000, 1.0 / L, lam=0.0, theta=th, restart=False)
    assert np.linalg.norm(x_nr.ravel() - xls) > 1e3 * np.linalg.norm(x.ravel() - xls)


def test_first_step_is_a_gradient_step_from_zero():
    N, A, D = 8, 6, 14
    th = oracle.default_angles(A)
    b = RNG.standard_normal((1, A, D))
    step = 1e-3
    x1 = oracle.mbir_solve(b, None, N, 1, step, lam=0.0, theta=th)
    # at x = 0 the gradient is -A^T b
    assert np.abs(x1 - step * oracle.radon_adj(b, N, th)).max() < 1e-14


def test_objective_decreases_with_prior():
    N, A, D = 16, 12, 24
    th = oracle.default_angles(A)
    xt = np.zeros((1, N, N))
    xt[0, 4:12, 5:11] = 1.0
    b = oracle.radon_fwd(xt, A, D, th)
    lam = 1e-3
    L = 1.05 * oracle.power_norm(N, A, D, None, RNG.standard_normal((1, N, N)), 30, th) \
        + lam * oracle.prior_lipschitz()
    x, log = oracle.mbir_solve(b, None, N, 60, 1.0 / L, lam=lam, theta=th, dims=2, return_log=True)
    G, H, _ = oracle.objective_grad(x, b, None, lam, oracle.PAPER_PRIOR, 2, th)
    G0, H0, _ = oracle.objective_grad(np.zeros_like(x), b, None, lam, oracle.PAPER_PRIOR, 2, th)
    assert G + H < 0.2 * (G0 + H0)
    assert math.isfinite(G + H)


def test_monotone_variant_converges_to_least_squares_monotonically():
    """Function-value restart (restart="monotone"): Phi(x_k) never increases
    and the iterates reach the dense least-squares solution, up to where the
    decrease of a gradient step, (step/2) |grad Phi|^2, falls below the FP64
    rounding of Phi itself (|x - x*| ~ sqrt(eps Phi* / lambda_min): here about
    1e-7 relative); the gradient test has no such floor."""
    N, A, D = 8, 24, 14
    th, M = _tiny(N, A, D)
    xt = RNG.standard_normal((N, N))
    b = (M @ xt.ravel()).reshape(1, A, D) + 0.01 * RNG.standard_normal((1, A, D))
    xls = np.linalg.lstsq(M, b.ravel(), rcond=None)[0]
    L = np.linalg.norm(M, 2) ** 2
    x, log = oracle.mbir_solve(b, None, N, 4000, 1.0 / L, lam=0.0, theta=th,
                               restart="monotone", return_log=True)
    assert np.linalg.norm(x.ravel() - xls) <= 1e-6 * np.linalg.norm(xls)
    # before that floor it keeps pace with the gradient-restart schedule
    x1k = oracle.mbir_solve(b, None, N, 1000, 1.0 / L, lam=0.0, theta=th, restart="monotone")
    x1g = oracle.mbir_solve(b, None, N, 1000, 1.0 / L, lam=0.0, theta=th, restart=True)
    e1k, e1g = (np.linalg.norm(v.ravel() - xls) for v in (x1k, x1g))
    assert e1k <= 1.5 * e1g
    phis = [e["phi_x"] for e in log]
    assert all(b2 <= b1 for b1, b2 in zip(phis, phis[1:]))
    assert any(e["restart"] for e in log)
    # the recorded value is the objective at the returned iterate
    r = M @ x.ravel() - b.ravel()
    assert abs(phis[-1] - 0.5 * float(r @ r)) <= 1e-12 * max(1.0, phis[-1])


def test_monotone_variant_rejects_a_step_that_raises_the_objective():
    """A step far above 1/L along the leading singular direction overshoots:
    the monotone variant keeps x_k (bitwise) and resets the momentum."""
    N, A, D = 8, 24, 14
    th, M = _tiny(N, A, D)
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    b = (S[0] * U[:, 0]).reshape(1, A, D)      # b = M v_1
    L = S[0] ** 2
    x, log = oracle.mbir_solve(b, None, N, 3, 10.0 / L, lam=0.0, theta=th,
                               restart="monotone", return_log=True)
    assert all(e["restart"] for e in log)
    assert np.array_equal(x, np.zeros_like(x))
    assert log[-1]["phi_x"] == 0.5 * float(np.sum(b * b))
    # with a safe step the first iterate is the plain gradient step, as in the other modes
    x1m = oracle.mbir_solve(b, None, N, 1, 1.0 / L, lam=0.0, theta=th, restart="monotone")
    x1g = oracle.mbir_solve(b, None, N, 1, 1.0 / L, lam=0.0, theta=th, restart=True)
    assert np.array_equal(x1m, x1g)


def test_monotone_variant_with_prior_and_weights():
    N, A, D = 16, 12, 24
    th = oracle.default_angles(A)
    xt = np.zeros((2, N, N))
    xt[:, 4:12, 5:11] = 1.0
    b = oracle.radon_fwd(xt, A, D, th) + 0.05 * RNG.standard_normal((2, A, D))
    w = RNG.uniform(0.3, 1.0, b.shape)
    lam = 2e-3
    L = 1.05 * oracle.power_norm(N, A, D, w, RNG.standard_normal((2, N, N)), 30, th) \
        + lam * oracle.prior_lipschitz()
    x, log = oracle.mbir_solve(b, w, N, 25, 1.0 / L, lam=lam, theta=th, dims=3,
                               restart="monotone", return_log=True)
    phis = [e["phi_x"] for e in log]
    assert all(b2 <= b1 for b1, b2 in zip(phis, phis[1:]))
    G, Hl = oracle.objective_value(x, b, w, lam, oracle.PAPER_PRIOR, 3, th)
    assert abs(phis[-1] - (G + Hl)) <= 1e-12 * phis[-1]
    G0, H0 = oracle.objective_value(np.zeros_like(x), b, w, lam, oracle.PAPER_PRIOR, 3, th)
    assert phis[-1] < 0.2 * (G0 + H0)


def test_continuing_from_a_state_equals_the_uninterrupted_iteration():
    """An iteration continued from (x_k, z_k, t_k) follows the uninterrupted
    one: z_k is rebuilt from x_k, x_{k-1} and the logged t values by the
    momentum rule, and two more iterations from there land on x_{k+2}
    (rounding aside).  A high starting t makes the gradient test restart
    early, so the continuation also carries a restart."""
    N, A, D = 8, 10, 14
    th, M = _tiny(N, A, D)
    b = np.random.default_rng(0).standard_normal((1, A, D))
    lam, k = 1e-3, 5  # from t = 20 this data restarts at the seventh iteration (index 6)
    step = 1.0 / (1.05 * np.linalg.eigvalsh(M.T @ M).max() + lam * oracle.prior_lipschitz())
    kw = dict(lam=lam, prior=oracle.PAPER_PRIOR, dims=2, theta=th, return_log=True)
    z0 = np.zeros((1, N, N))
    x_all, log_all = oracle.mbir_solve(b, None, N, k + 2, step, z0=z0, t0=20.0, **kw)
    x_km1, _ = oracle.mbir_solve(b, None, N, k - 1, step, z0=z0, t0=20.0, **kw)
    x_k, log_k = oracle.mbir_solve(b, None, N, k, step, z0=z0, t0=20.0, **kw)
    t_prev = log_k[-2]["t"]  # t_{k-1} as used for z_k, unless iteration k restarted
    if log_k[-1]["restart"]:
        t_prev = 1.0
    t_k = log_k[-1]["t"]
    z_k = x_k + ((t_prev - 1.0) / t_k) * (x_k - x_km1)
    x_cont, log_cont = oracle.mbir_solve(b, None, N, 2, step, x0=x_k, z0=z_k, t0=t_k, **kw)
    assert any(e["restart"] for e in log_all)
    assert [e["restart"] for e in log_cont] == [e["restart"] for e in log_all[k:]]
    assert np.abs(x_cont - x_all).max() <= 1e-12 * max(1.0, np.abs(x_all).max())
