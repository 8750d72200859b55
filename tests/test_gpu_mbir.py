"""Parity of the CUDA MBIR path (gradient, prior, power iteration, solver)
with the FP64 oracle, through the C ABI.

Tolerances: objective gradient relative L2 <= 1e-4 (A and A^T are each within
~2e-6 of exact, the prior is FP32); power-iteration eigenvalue <= 1e-5
relative; volume after the fixed iteration count <= 1e-3 relative L2.
"""
import numpy as np
import pytest

import oracle
from paper_2304_12934_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_12934_gb300 import api as a
    a.load()
    return a


def t32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda:0")


def np64(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


N, A, D = 128, 90, 184


def _data(B, seed0=synth.BASE_SEED):
    ells = [synth.random_ellipses(N, seed0 + k) for k in range(B)]
    f = np.stack([synth.rasterize(N, e) for e in ells])
    b = np.stack([synth.ellipse_line_integrals(e, oracle.default_angles(A), D) for e in ells])
    return f.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("dims", [2, 3])
def test_gradient_and_objective_match_oracle(api, dims):
    B = 3
    f, b = _data(B)
    rng = np.random.default_rng(dims)
    w = rng.uniform(0.2, 1.0, b.shape).astype(np.float32).astype(np.float64)
    b = 0.5 * b
    prior = api.Prior(lam=2e-3, dims=dims)
    with api.Plan(N, A, D, max_batch=2) as plan:
        g, obj = api.mbir_grad(plan, t32(f), t32(b), t32(w), prior)
        gn, objn = api.mbir_grad(plan, t32(f), t32(b), t32(w), None)
        # zero weights remove the data term exactly: the prior gradient alone
        gp, objp = api.mbir_grad(plan, t32(f), t32(b), t32(np.zeros_like(w)), prior)
    pd = dict(p=prior.p, sigma=prior.sigma, c=prior.c)
    G, H, go = oracle.objective_grad(f, b, w, prior.lam, pd, dims)
    assert rel(np64(g), go) <= 1e-4
    o = obj.cpu().numpy()
    assert abs(o[0] - G) <= 1e-5 * G
    assert abs(o[1] - H) <= 1e-5 * H
    # the prior part alone
    Hv, gh = oracle.prior_value_grad(f, dims, **pd)
    assert rel(np64(gp), prior.lam * gh) <= 1e-5
    assert float(objp.cpu().numpy()[0]) == 0.0
    assert abs(float(objp.cpu().numpy()[1]) - prior.lam * Hv) <= 1e-5 * prior.lam * Hv
    assert float(objn.cpu().numpy()[1]) == 0.0
    Gn, _, gno = oracle.objective_grad(f, b, w, 0.0, pd, dims)
    assert rel(np64(gn), gno) <= 2e-5


def test_power_norm_matches_oracle(api):
    B = 1
    rng = np.random.default_rng(21)
    v0 = synth.random_start((B, N, N), 99).astype(np.float32).astype(np.float64)
    w = rng.uniform(0.2, 1.0, (B, A, D)).astype(np.float32).astype(np.float64)
    lo = oracle.power_norm(N, A, D, w, v0, 20)
    with api.Plan(N, A, D) as plan:
        lg = api.mbir_power_norm(plan, t32(v0), t32(w), n_iter=20)
    assert abs(lg - lo) <= 1e-5 * lo


def _step(lam_prior):
    v0 = synth.random_start((1, N, N), 7)
    L = 1.05 * oracle.power_norm(N, A, D, None, v0, 30)
    return 1.0 / (L + 8.0 * lam_prior / ((1 / 0.7) ** 2 * 1e-4))


def test_solver_matches_oracle_after_20_iterations(api):
    f, b = _data(1)
    lam = 1e-3
    step = _step(lam)
    prior = api.Prior(lam=lam, dims=2)
    xo, log = oracle.mbir_solve(b, None, N, 20, step, lam=lam,
                                prior=dict(p=prior.p, sigma=prior.sigma, c=prior.c),
                                dims=2, return_log=True)
    with api.Plan(N, A, D) as plan:
        x = torch.zeros((1, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), None, x, 20, step, prior)
    assert st.k == 20
    assert st.n_restarts == sum(e["restart"] for e in log)
    assert rel(np64(x), xo) <= 1e-3


def test_solver_noisy_weighted_3d(api):
    """Poisson data with weights and the 26-neighbour prior, 10 iterations."""
    B = 2
    ells = [synth.random_ellipses(N, synth.BASE_SEED + k, scale=1.0 / N) for k in range(B)]
    th = oracle.default_angles(A)
    p = np.stack([synth.ellipse_line_integrals(e, th, D) for e in ells])
    b, w = synth.poisson_measurement(p, 1e4, 5)
    b = b.astype(np.float32).astype(np.float64)
    w = w.astype(np.float32).astype(np.float64)
    lam = 1e-2
    v0 = synth.random_start((B, N, N), 3)
    L = 1.05 * oracle.power_norm(N, A, D, w, v0, 30)
    step = 1.0 / (L + 8.0 * lam / ((1 / 0.7) ** 2 * 1e-4))
    prior = api.Prior(lam=lam, dims=3)
    xo = oracle.mbir_solve(b, w, N, 10, step, lam=lam,
                           prior=dict(p=prior.p, sigma=prior.sigma, c=prior.c), dims=3)
    with api.Plan(N, A, D, max_batch=1) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        api.mbir_solve(plan, t32(b), t32(w), x, 10, step, prior)
    assert rel(np64(x), xo) <= 1e-3


def test_resume_equals_uninterrupted_bitwise(api):
    f, b = _data(2)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=2)
    with api.Plan(N, A, D, max_batch=2) as plan:
        bt = t32(b)
        x1 = torch.zeros((2, N, N), device="cuda:0")
        api.mbir_solve(plan, bt, None, x1, 20, step, prior)
        x2 = torch.zeros((2, N, N), device="cuda:0")
        st = api.mbir_solve(plan, bt, None, x2, 10, step, prior)
        # checkpoint the state to host and back, then resume
        z_host, t, k, nr = st.z.cpu(), st.t, st.k, st.n_restarts
        st2 = api.SolveState(x2)
        st2.z.copy_(z_host)
        st2.t, st2.k, st2.n_restarts = t, k, nr
        api.mbir_solve(plan, bt, None, x2, 10, step, prior, state=st2)
    assert st2.k == 20
    assert torch.equal(x1, x2)


def test_host_buffer_solve_matches_device_solve(api):
    f, b = _data(1)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=2)
    with api.Plan(N, A, D) as plan:
        x = torch.zeros((1, N, N), device="cuda:0")
        api.mbir_solve(plan, t32(b), None, x, 5, step, prior)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        xh = torch.zeros((1, N, N), dtype=torch.float32).pin_memory()
        api.mbir_solve_host(plan, bh, None, xh, 5, step, prior)
    assert torch.equal(xh, x.cpu())


@pytest.mark.parametrize("n_iter", [4, 1])
def test_host_streamed_solve_in_slabs_matches_device_solve(api, n_iter):
    """Five slices copied in slabs of two on the copy stream, weights and the
    3D prior: identical to the same solve on resident device buffers.  The last
    iteration returns x slab by slab while later slabs still compute (with
    n_iter = 1 that iteration also waits for the inbound slabs)."""
    B = 5
    f, b = _data(B)
    rng = np.random.default_rng(9)
    w = rng.uniform(0.5, 1.0, b.shape)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=3)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        sd = api.mbir_solve(plan, t32(b), t32(w), x, n_iter, step, prior)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        wh = torch.tensor(w, dtype=torch.float32).pin_memory()
        xh = torch.zeros((B, N, N), dtype=torch.float32).pin_memory()
        sh = api.mbir_solve_host(plan, bh, wh, xh, n_iter, step, prior)
    assert torch.equal(xh, x.cpu())
    assert sh.k == sd.k == n_iter and sh.n_restarts == sd.n_restarts
    assert torch.equal(sh.z.cpu(), sd.z.cpu())
    assert abs(sh.obj[0] - sd.obj[0]) <= 1e-12 * abs(sd.obj[0])
    assert abs(sh.obj[1] - sd.obj[1]) <= 1e-9 * abs(sd.obj[1])


@pytest.mark.parametrize("dims", [3, 2])
def test_prior_on_a_tall_volume_matches_oracle(api, dims):
    """150 slices of 128^2: tiles inside the volume and at its border, and
    z marches long enough for every level of the per-thread FP32 -> FP64
    accumulation of H.  Zero data weights leave the prior term alone."""
    g, h, go, ho = _tall_prior_case(api, dims)
    assert rel(g, go) <= 1e-5
    assert abs(h - ho) <= 1e-5 * ho


def _tall_prior_case(api, dims):
    B, n = 150, 128
    rng = np.random.default_rng(77 + dims)
    base = synth.rasterize(n, synth.random_ellipses(n, synth.BASE_SEED + 9))
    f = np.repeat(base[None], B, axis=0) * np.linspace(0.5, 1.5, B)[:, None, None]
    f[::7] += 0.05 * rng.standard_normal((len(f[::7]), n, n))   # flat regions and noisy slices
    f = f.astype(np.float32).astype(np.float64)
    b = np.zeros((B, 8, 184))
    prior = api.Prior(lam=1e-3, dims=dims)
    with api.Plan(n, 8, 184, max_batch=B) as plan:
        g, obj = api.mbir_grad(plan, t32(f), t32(b), t32(np.zeros_like(b)), prior)
    pd = dict(p=prior.p, sigma=prior.sigma, c=prior.c)
    Hv, gh = oracle.prior_value_grad(f, dims, **pd)
    return np64(g), float(obj.cpu().numpy()[1]), prior.lam * gh, prior.lam * Hv


# ------------------------------------------------- monotone variant (NEXT) ----
def _noisy_weighted(B=2):
    ells = [synth.random_ellipses(N, synth.BASE_SEED + 40 + k, scale=1.0 / N) for k in range(B)]
    th = oracle.default_angles(A)
    p = np.stack([synth.ellipse_line_integrals(e, th, D) for e in ells])
    b, w = synth.poisson_measurement(p, 1e4, 15)
    return b.astype(np.float32).astype(np.float64), w.astype(np.float32).astype(np.float64)


def test_monotone_solver_matches_oracle(api):
    """Function-value test (Sec. 3 reading): 20 iterations on weighted noisy
    data with the 26-neighbour prior against the oracle's monotone schedule;
    the reported objective is the one at the returned x."""
    b, w = _noisy_weighted(2)
    lam = 1e-2
    v0 = synth.random_start((2, N, N), 3)
    step = 1.0 / (1.05 * oracle.power_norm(N, A, D, w, v0, 30) + 8.0 * lam / ((1 / 0.7) ** 2 * 1e-4))
    prior = api.Prior(lam=lam, dims=3)
    pd = dict(p=prior.p, sigma=prior.sigma, c=prior.c)
    xo, log = oracle.mbir_solve(b, w, N, 20, step, lam=lam, prior=pd, dims=3,
                                restart="monotone", return_log=True)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((2, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), t32(w), x, 20, step, prior, restart="monotone")
    assert st.k == 20
    assert rel(np64(x), xo) <= 1e-3
    G, Hl = oracle.objective_value(np64(x), b, w, lam, pd, 3)
    assert abs(st.obj[0] - G) <= 1e-5 * G and abs(st.obj[1] - Hl) <= 1e-5 * Hl
    assert abs(sum(st.obj) - log[-1]["phi_x"]) <= 1e-4 * log[-1]["phi_x"]


def test_monotone_objective_never_increases_and_resumes_bitwise(api):
    b, w = _noisy_weighted(2)
    lam = 1e-2
    v0 = synth.random_start((2, N, N), 4)
    step = 1.0 / (1.05 * oracle.power_norm(N, A, D, w, v0, 30) + 8.0 * lam / ((1 / 0.7) ** 2 * 1e-4))
    prior = api.Prior(lam=lam, dims=3)
    with api.Plan(N, A, D, max_batch=2) as plan:
        bt, wt = t32(b), t32(w)
        x1 = torch.zeros((2, N, N), device="cuda:0")
        api.mbir_solve(plan, bt, wt, x1, 12, step, prior, restart="monotone")
        x2 = torch.zeros((2, N, N), device="cuda:0")
        st = api.SolveState(x2)
        phis = []
        for _ in range(12):   # one iteration per call: Phi(x_k) is recomputed each time
            api.mbir_solve(plan, bt, wt, x2, 1, step, prior, restart="monotone", state=st)
            phis.append(sum(st.obj))
    assert st.k == 12
    assert all(p2 <= p1 for p1, p2 in zip(phis, phis[1:]))
    assert torch.equal(x1, x2)


def test_monotone_rejects_an_overshooting_step(api):
    """A step 1000 times 1/L raises the objective: x stays at its start
    (bitwise), every step is rejected and counted as a restart."""
    f, b = _data(1)
    L = 1.0 / _step(0.0)
    with api.Plan(N, A, D) as plan:
        x = torch.zeros((1, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), None, x, 3, 1000.0 / L, None, restart="monotone")
    assert st.n_restarts == 3
    assert torch.count_nonzero(x) == 0
    assert abs(st.obj[0] - 0.5 * float(np.sum(b * b))) <= 1e-5 * 0.5 * float(np.sum(b * b))
    assert st.obj[1] == 0.0
