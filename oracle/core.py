"""FP64 oracle: ctypes binding of radon_oracle.c, prior, MBIR loop.

TEST INFRASTRUCTURE ONLY (see package docstring).  Every routine is a plain
restatement of the paper's definitions:

* Radon operator A and adjoint A^T: Sec. 2.1 Eq. radon_transform / line_eqn,
  Sec. 2.2 Eqs. fourier_sum and nufft (exact sums, no gridding), Sec. 3
  Eq. transpose.  Implemented in C (``radon_oracle.c``).
* Objective: Sec. 3 Eq. objfn with the data term read as 1/2 ||Af - b||_W^2 so
  that its gradient is Eq. gradient's A^T (Af - b) (weighted by W).
* Prior: Sec. 3 Eqs. reg2/reg3 (qGGMRF over the 1-hop neighbourhood), with the
  paper's hyper-parameters p=1.2, sigma=1/0.7, c=1e-4 (Sec. 5).
* Optimizer: Sec. 3 last paragraph (an accelerated gradient method that is
  monotone and restarts), read as FISTA with a constant step and the gradient
  restart test.  This schedule is parity unpinned by the paper beyond the invariants
  tested in tests/test_oracle_mbir.py.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

__all__ = [
    "build", "lib", "default_angles", "radon_fwd", "radon_adj",
    "radon_fwd_at", "radon_adj_at", "dirichlet", "neighbour_offsets",
    "prior_weights", "rho", "rho_prime", "prior_value_grad", "data_grad",
    "objective_grad", "objective_value", "power_norm", "prior_lipschitz", "mbir_solve",
    "normal_op", "PAPER_PRIOR",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radon_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_radon.so")

# Sec. 5 hyper-parameters of the prior: p 1.2, sigma 1/0.7, c 1e-4
PAPER_PRIOR = dict(p=1.2, sigma=1.0 / 0.7, c=1e-4)


def build(force: bool = False) -> str:
    """Compile radon_oracle.c into a shared object (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        d = ctypes.c_double
        L.oracle_radon_fwd.argtypes = [i, i, i, dp, dp, dp]
        L.oracle_radon_adj.argtypes = [i, i, i, dp, dp, dp]
        L.oracle_radon_fwd_batch.argtypes = [i, i, i, i, dp, d, dp, dp]
        L.oracle_radon_adj_batch.argtypes = [i, i, i, i, dp, d, dp, dp]
        L.oracle_radon_fwd_at_shift.argtypes = [i, i, i, dp, d, dp, i, ip, ip, dp]
        L.oracle_radon_adj_at_shift.argtypes = [i, i, i, dp, d, dp, i, ip, dp]
        L.oracle_dirichlet.argtypes = [i, ctypes.c_double]
        L.oracle_dirichlet.restype = ctypes.c_double
        for fn in ("oracle_radon_fwd", "oracle_radon_adj", "oracle_radon_fwd_batch",
                   "oracle_radon_adj_batch", "oracle_radon_fwd_at_shift", "oracle_radon_adj_at_shift"):
            getattr(L, fn).restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_angles(n_angles: int) -> np.ndarray:
    """theta_a = a*pi/A, a = 0..A-1: uniform over [0, pi) (Sec. 2.1)."""
    return np.arange(n_angles, dtype=np.float64) * (math.pi / n_angles)


def _theta(theta, n_angles):
    th = default_angles(n_angles) if theta is None else np.ascontiguousarray(theta, np.float64)
    assert th.shape == (n_angles,)
    return th


def radon_fwd(f: np.ndarray, n_angles: int, n_det: int, theta=None, delta: float = 0.0) -> np.ndarray:
    """y = A f for f of shape [N,N] or [B,N,N]; returns [A,D] or [B,A,D].
    delta: rotation-axis offset (detector coordinate of the axis minus D/2)."""
    f = np.ascontiguousarray(f, np.float64)
    squeeze = f.ndim == 2
    if squeeze:
        f = f[None]
    B, N, N2 = f.shape
    assert N == N2
    th = _theta(theta, n_angles)
    y = np.zeros((B, n_angles, n_det), np.float64)
    rc = lib().oracle_radon_fwd_batch(B, N, n_angles, n_det, _dp(th), float(delta), _dp(f), _dp(y))
    if rc:
        raise ValueError(f"oracle_radon_fwd failed: {rc}")
    return y[0] if squeeze else y


def radon_adj(y: np.ndarray, n: int, theta=None, delta: float = 0.0) -> np.ndarray:
    """x = A^T y for y of shape [A,D] or [B,A,D]; returns [N,N] or [B,N,N]."""
    y = np.ascontiguousarray(y, np.float64)
    squeeze = y.ndim == 2
    if squeeze:
        y = y[None]
    B, A, D = y.shape
    th = _theta(theta, A)
    x = np.zeros((B, n, n), np.float64)
    rc = lib().oracle_radon_adj_batch(B, n, A, D, _dp(th), float(delta), _dp(y), _dp(x))
    if rc:
        raise ValueError(f"oracle_radon_adj failed: {rc}")
    return x[0] if squeeze else x


def radon_fwd_at(f, n_angles, n_det, a_idx, i_idx, theta=None, delta: float = 0.0) -> np.ndarray:
    """Sampled entries y(a_k, i_k) of A f (single slice), Dirichlet closed form."""
    f = np.ascontiguousarray(f, np.float64)
    N = f.shape[0]
    th = _theta(theta, n_angles)
    a_idx = np.ascontiguousarray(a_idx, np.int32)
    i_idx = np.ascontiguousarray(i_idx, np.int32)
    out = np.zeros(a_idx.shape[0], np.float64)
    rc = lib().oracle_radon_fwd_at_shift(N, n_angles, n_det, _dp(th), float(delta), _dp(f),
                                         out.shape[0], _ip(a_idx), _ip(i_idx), _dp(out))
    if rc:
        raise ValueError(f"oracle_radon_fwd_at failed: {rc}")
    return out


def radon_adj_at(y, n, pix_idx, theta=None, delta: float = 0.0) -> np.ndarray:
    """Sampled pixels x(pix_k) of A^T y (single slice), Dirichlet closed form."""
    y = np.ascontiguousarray(y, np.float64)
    A, D = y.shape
    th = _theta(theta, A)
    pix_idx = np.ascontiguousarray(pix_idx, np.int32)
    out = np.zeros(pix_idx.shape[0], np.float64)
    rc = lib().oracle_radon_adj_at_shift(n, A, D, _dp(th), float(delta), _dp(y), out.shape[0],
                                         _ip(pix_idx), _dp(out))
    if rc:
        raise ValueError(f"oracle_radon_adj_at failed: {rc}")
    return out


def normal_op(f: np.ndarray, n_angles: int, n_det: int, theta=None, delta: float = 0.0) -> np.ndarray:
    """A^T A f for f of shape [N,N] or [B,N,N]: the Hessian of the unweighted data
    term (Sec. 3 Eqs. gradient, transpose), as the plain composition of the exact
    operators above."""
    n = f.shape[-1]
    return radon_adj(radon_fwd(f, n_angles, n_det, theta, delta), n, theta, delta)


def dirichlet(D: int, u: float) -> float:
    return lib().oracle_dirichlet(D, float(u))


# ---------------------------------------------------------------- prior ----
def neighbour_offsets(dims: int):
    """1-hop neighbourhood {n : ||m - n||_inf <= 1, n != m} (Sec. 3 Eq. reg2).

    dims=2: the 8 in-plane neighbours (offsets in (z, y, x) with z = 0);
    dims=3: all 26 neighbours of the voxel grid.
    """
    offs = []
    zr = (-1, 0, 1) if dims == 3 else (0,)
    for dz in zr:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) != (0, 0, 0):
                    offs.append((dz, dy, dx))
    return offs


def prior_weights(dims: int):
    """w_mn proportional to 1/||m-n||_2 and summing to one over the
    neighbourhood (Sec. 3, the sentence after Eq. reg3)."""
    offs = neighbour_offsets(dims)
    inv = np.array([1.0 / math.sqrt(dz * dz + dy * dy + dx * dx) for dz, dy, dx in offs])
    return offs, inv / inv.sum()


def rho(delta, p, sigma, c):
    """h_mn of Sec. 3 Eq. reg3 as a function of delta = f_m - f_n."""
    u = np.abs(delta) / sigma
    return u * u / (c + u ** (2.0 - p))


def rho_prime(delta, p, sigma, c):
    """d rho / d delta, differentiated by hand from Eq. reg3."""
    u = np.asarray(delta, np.float64) / sigma
    au = np.abs(u)
    q = au ** (2.0 - p)
    return (u / sigma) * (2.0 * c + p * q) / (c + q) ** 2


def _pair_slices(shape, off):
    """Slices (sl_m, sl_n) selecting every in-bounds pair n = m + off."""
    sm, sn = [], []
    for L, d in zip(shape, off):
        if d >= 0:
            sm.append(slice(0, L - d))
            sn.append(slice(d, L))
        else:
            sm.append(slice(-d, L))
            sn.append(slice(0, L + d))
    return tuple(sm), tuple(sn)


def prior_value_grad(f, dims=2, p=1.2, sigma=1.0 / 0.7, c=1e-4):
    """H(f) = sum_m sum_{n in N(m)} w_mn rho(f_m - f_n) and its gradient.

    f has shape [B, N, N] (slices along z).  Neighbours outside the volume are
    left out and the weights are not renormalised.  Every ordered pair (m, n)
    is one term, as written in Eq. reg2; the gradient differentiates each term
    with respect to both of its pixels.
    """
    f = np.asarray(f, np.float64)
    if f.ndim == 2:
        f = f[None]
        squeeze = True
    else:
        squeeze = False
    offs, w = prior_weights(dims)
    H = 0.0
    g = np.zeros_like(f)
    for off, wd in zip(offs, w):
        sm, sn = _pair_slices(f.shape, off)
        delta = f[sm] - f[sn]
        H += wd * float(rho(delta, p, sigma, c).sum())
        rp = wd * rho_prime(delta, p, sigma, c)
        g[sm] += rp
        g[sn] -= rp
    return H, (g[0] if squeeze else g)


def prior_lipschitz(p=1.2, sigma=1.0 / 0.7, c=1e-4):
    """Bound on ||Hessian of H||: 4 * rho''(0) = 8 / (sigma^2 c).

    rho''(0) = 2/(sigma^2 c) is the largest curvature of Eq. reg3 for
    1 <= p <= 2; the neighbourhood Laplacian with unit-sum weights has norm
    at most 2, and every pair appears twice in Eq. reg2.
    """
    return 8.0 / (sigma * sigma * c)


# ----------------------------------------------------------------- MBIR ----
def data_grad(f, b, wt, theta=None):
    """Data term G = 1/2 sum W (A f - b)^2 and its gradient A^T W (A f - b)."""
    B, N, _ = f.shape
    _, A, D = b.shape
    r = radon_fwd(f, A, D, theta) - b
    if wt is not None:
        wr = wt * r
    else:
        wr = r
    G = 0.5 * float(np.sum(wr * r))
    return G, radon_adj(wr, N, theta)


def objective_grad(f, b, wt, lam, prior, dims, theta=None):
    """Phi(f) = G(f) + lam H(f) and its gradient (Sec. 3 Eqs. objfn, gradient)."""
    G, g = data_grad(f, b, wt, theta)
    if lam != 0.0:
        H, gh = prior_value_grad(f, dims, **prior)
        return G, lam * H, g + lam * gh
    return G, 0.0, g


def objective_value(f, b, wt, lam, prior, dims, theta=None):
    """(G(f), lam H(f)) without the gradient (Sec. 3 Eq. objfn)."""
    B, N, _ = f.shape
    _, A, D = b.shape
    r = radon_fwd(f, A, D, theta) - b
    G = 0.5 * float(np.sum((wt * r if wt is not None else r) * r))
    Hl = lam * prior_value_grad(f, dims, **prior)[0] if lam != 0.0 else 0.0
    return G, Hl


def power_norm(n, n_angles, n_det, wt, v0, n_iter, theta=None):
    """Largest eigenvalue of A^T W A by power iteration from the given start.

    v_0 = v0/||v0||; each step u = A^T W A v, lambda = <v, u>, v = u/||u||.
    Returns the last Rayleigh quotient.
    """
    v = np.asarray(v0, np.float64).copy()
    v /= np.linalg.norm(v)
    lam = 0.0
    A, D = n_angles, n_det
    for _ in range(n_iter):
        y = radon_fwd(v, A, D, theta)
        if wt is not None:
            y = wt * y
        u = radon_adj(y, n, theta)
        lam = float(np.sum(v * u))
        v = u / np.linalg.norm(u)
    return lam


def mbir_solve(b, wt, n, n_iter, step, lam=1.0, prior=None, dims=2,
               theta=None, x0=None, restart=True, return_log=False, z0=None, t0=1.0):
    """Accelerated gradient on Phi = G + lam H (Sec. 3), from x_0 = z_0 = x0
    (zero by default) with t_0 = 1; all scalars FP64.  z0 and t0 continue an
    iteration from a given state (x_k, z_k, t_k) instead: x_0 = x0, z_0 = z0.

    Reading of the end of Sec. 3 (accelerated gradient, monotone, with restart):
        v       = z_k - step * grad Phi(z_k)
        restart = True (gradient restart):
            x_{k+1} = v; restart (t_k := 1) if <grad Phi(z_k), x_{k+1} - x_k> > 0
        restart = "monotone" (function-value test):
            x_{k+1} = v if Phi(v) <= Phi(x_k), else x_{k+1} = x_k and t_k := 1,
            so Phi(x_k) never increases
        restart = False: x_{k+1} = v, no restart (plain FISTA)
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        z_{k+1} = x_{k+1} + ((t_k - 1)/t_{k+1}) (x_{k+1} - x_k)
    """
    prior = PAPER_PRIOR if prior is None else prior
    monotone = restart == "monotone"
    B = b.shape[0]
    x = np.zeros((B, n, n)) if x0 is None else np.asarray(x0, np.float64).copy()
    z = x.copy() if z0 is None else np.asarray(z0, np.float64).copy()
    t = float(t0)
    phi_x = sum(objective_value(x, b, wt, lam, prior, dims, theta)) if monotone else None
    log = []
    for k in range(n_iter):
        G, Hl, g = objective_grad(z, b, wt, lam, prior, dims, theta)
        v = z - step * g
        dot = float(np.sum(g * (v - x)))
        if monotone:
            Gv, Hv = objective_value(v, b, wt, lam, prior, dims, theta)
            accepted = Gv + Hv <= phi_x
            restarted = not accepted
            x_new = v if accepted else x.copy()
            if accepted:
                phi_x = Gv + Hv
        else:
            restarted = bool(restart and dot > 0.0)
            x_new = v
        if restarted:
            t = 1.0
        t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_new
        z = x_new + beta * (x_new - x)
        x = x_new
        t = t_new
        entry = dict(k=k, data=G, prior=Hl, dot=dot, restart=restarted, t=t)
        if monotone:
            entry["phi_x"] = phi_x
        log.append(entry)
    return (x, log) if return_log else x
