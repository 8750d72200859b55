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


@pytest.mark.parametrize("restart", [True, False])
def test_fused_momentum_point_across_calls_and_restarts(api, restart):
    """Every iteration with a prior makes z_{k+1} inside the prior pass (a copy
    of x_{k+1} after a restart), and the state's z and g buffers exchange roles
    each iteration.  One call of 13 iterations and 13 calls of one iteration
    (the exchange handed back through the state) give the same x, z, t and
    restart count, bit for bit.  Both resume from x = z = 0 with momentum
    t = 20, from which the gradient test restarts (at the fourth iteration in
    the FP64 oracle), so both branches of the check-and-copy run; the result
    matches the oracle's iteration from the same state to 1e-3."""
    f, b = _data(2)
    lam = 1e-3
    step = _step(lam)
    prior = api.Prior(lam=lam, dims=3)
    n = 13
    xo, log = oracle.mbir_solve(b, None, N, n, step, lam=lam, prior=dict(p=prior.p, sigma=prior.sigma, c=prior.c),
                                dims=3, restart=restart, return_log=True, z0=np.zeros((2, N, N)), t0=20.0)
    with api.Plan(N, A, D, max_batch=2) as plan:
        bt = t32(b)
        out = []
        for single in (False, True):
            x = torch.zeros((2, N, N), device="cuda:0")
            st = api.SolveState(x)
            st.z.zero_()
            st.t, st.k = 20.0, 1
            for _ in range(n if single else 1):
                api.mbir_solve(plan, bt, None, x, 1 if single else n, step, prior, restart=restart, state=st)
            out.append((x, st))
    (x1, st1), (x2, st2) = out
    assert st1.k == st2.k == n + 1
    assert st1.n_restarts == st2.n_restarts == sum(e["restart"] for e in log)
    if restart:
        assert st1.n_restarts > 0
    assert torch.equal(x1, x2)
    assert torch.equal(st1.z, st2.z)
    assert st1.t == st2.t
    assert rel(np64(x1), xo) <= 1e-3


def test_special_function_unit_probe(api):
    """The measured lg2 / ex2 / rcp rates behind the prior kernel's roofline:
    positive, at least one lane operation per clock and SM at 1 GHz (all
    Blackwell parts run these at 16 lanes per clock and SM or more), and an
    unknown operation is rejected before any launch."""
    import ctypes
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for op in ("lg2", "ex2", "rcp"):
        r = api.sfu_throughput(op)
        assert r > sms * 1e9, (op, r)
    out = ctypes.c_double()
    assert api.load().tc_sfu_throughput(3, ctypes.byref(out), None) == -1
    assert api.load().tc_sfu_throughput(0, None, None) == -1


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


@pytest.mark.parametrize("n_iter", [3, 1])
def test_resumed_host_streamed_solve_matches_device_solve(api, n_iter):
    """A resumed solve from host buffers (z already on the device) starts each
    chunk's data gradient once the chunk's b and w have arrived, and each
    prior waits for its slab of x: identical to the resumed device solve."""
    B = 5
    f, b = _data(B)
    rng = np.random.default_rng(11)
    w = rng.uniform(0.5, 1.0, b.shape)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=3)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        sd = api.mbir_solve(plan, t32(b), t32(w), x, 2, step, prior)
        api.mbir_solve(plan, t32(b), t32(w), x, n_iter, step, prior, state=sd)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        wh = torch.tensor(w, dtype=torch.float32).pin_memory()
        xh = torch.zeros((B, N, N), dtype=torch.float32).pin_memory()
        dev = {}
        sh = api.mbir_solve_host(plan, bh, wh, xh, 2, step, prior, dev=dev)
        api.mbir_solve_host(plan, bh, wh, xh, n_iter, step, prior, state=sh, dev=dev)
    assert torch.equal(xh, x.cpu())
    assert sh.k == sd.k == 2 + n_iter and sh.n_restarts == sd.n_restarts
    assert torch.equal(sh.z.cpu(), sd.z.cpu())


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


# --------------------------------------- noisy 512^2 workload (stored oracle) ----
def test_noisy_512_weighted_solve_matches_oracle(api):
    """The noisy workload's geometry: one 512^2 slice, 180 angles, 724 bins,
    Poisson data at I0 = 1e4 with count weights (Sec. 5, b = -log(I/I0)),
    8-neighbour qGGMRF with lambda = 1e-2, gradient restart.  10 and 50
    iterations against the FP64 oracle's iterates stored by
    tests/golden/make_oracle_golden.py (same b, w and step): relative L2
    <= 1e-3 and the same number of restarts."""
    import make_oracle_golden as mk
    c = mk.NOISY
    ref = np.load(mk.noisy_path())
    prior = api.Prior(lam=c["lam"], dims=c["dims"])
    with api.Plan(c["N"], c["A"], c["D"], max_batch=1) as plan:
        b, w = t32(ref["b"]), t32(ref["w"])
        for iters, key, rkey in ((10, "x10", "restarts10"), (c["iters"], "x", "restarts")):
            x = torch.zeros((1, c["N"], c["N"]), device="cuda:0")
            st = api.mbir_solve(plan, b, w, x, iters, float(ref["step"]), prior)
            assert st.k == iters
            assert st.n_restarts == int(ref[rkey])
            err = rel(np64(x)[0], ref[key].astype(np.float64))
            assert err <= 1e-3, (iters, err)
        # the objective terms at the last gradient point z_49 of the 50-iteration solve
        assert abs(st.obj[0] - float(ref["data"][-1])) <= 1e-4 * float(ref["data"][-1])
        assert abs(st.obj[1] - float(ref["prior"][-1])) <= 1e-4 * float(ref["prior"][-1])


# ------------------------------------------------- step size in the library ----
def test_library_step_matches_oracle_step(api):
    """opts.step <= 0: the library derives 1/L, L = 1.05 lambda_max(A^T W A)
    + lambda 8/(sigma^2 c) (reading of Sec. 3), by power iteration over the
    batch.  Against the oracle's power iteration from its own start (both
    converged): relative 1e-5.  The host-streamed solve derives the same step
    bit for bit, and a resumed call reuses it."""
    # two copies of one slice: the block-diagonal normal operator keeps that
    # slice's (well separated) top eigenvalue, so both power iterations
    # converge; slices with different weights would put two nearly equal
    # eigenvalues on top and stall any power iteration
    B = 2
    _, b1 = _data(1)
    w1 = np.random.default_rng(44).uniform(0.3, 1.0, b1.shape).astype(np.float32).astype(np.float64)
    b, w = np.concatenate([b1, b1]), np.concatenate([w1, w1])
    lam = 1e-3
    prior = api.Prior(lam=lam, dims=3)
    v0 = synth.random_start((1, N, N), 45)
    L = 1.05 * oracle.power_norm(N, A, D, w1, v0, 40) + lam * oracle.prior_lipschitz(**oracle.PAPER_PRIOR)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), t32(w), x, 3, None, prior, power_iter=40)
        assert abs(st.step * L - 1.0) <= 1e-5, st.step * L
        x2 = torch.zeros((B, N, N), device="cuda:0")
        s2 = api.mbir_solve(plan, t32(b), t32(w), x2, 3, st.step, prior)
        assert torch.equal(x, x2)
        api.mbir_solve(plan, t32(b), t32(w), x, 2, None, prior, state=st)   # resumes with st.step
        api.mbir_solve(plan, t32(b), t32(w), x2, 2, None, prior, state=s2)
        assert torch.equal(x, x2)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        wh = torch.tensor(w, dtype=torch.float32).pin_memory()
        xh = torch.zeros((B, N, N), dtype=torch.float32).pin_memory()
        sh = api.mbir_solve_host(plan, bh, wh, xh, 3, None, prior, power_iter=40)
        assert sh.step == st.step
        with pytest.raises(api.TcError):   # a resumed state with no step to reuse
            bad = api.SolveState(x)
            bad.k = 1
            api.mbir_solve(plan, t32(b), t32(w), x, 1, None, prior, state=bad)


# ------------------------------------------------ the headline geometry ----
def _headline_inputs(B, dev):
    n, a, d = 2048, 128, 2896
    theta = oracle.default_angles(a)
    p = synth.ellipsoid_sinogram_torch(n, B, theta, d, dev, scale=1.0 / n, seed=synth.BASE_SEED + 77)
    b, w = synth.poisson_measurement_torch(p, 1e4, synth.BASE_SEED + 78)
    return n, a, d, b.contiguous(), w.contiguous()


def test_headline_first_iterate_matches_oracle(api):
    """2048^2, 128 angles, 2896 bins, Poisson weights, 26-neighbour prior: from
    x_0 = 0 the first iterate is x_1 = step A^T (W b) (the prior's gradient
    vanishes on a constant image).  1024 sampled pixels per slice against the
    oracle's closed-form adjoint: relative L2 <= 2e-5."""
    dev = torch.device("cuda:0")
    B = 2
    n, a, d, b, w = _headline_inputs(B, dev)
    step = 3.75e-6
    prior = api.Prior(lam=1e-2, dims=3)
    with api.Plan(n, a, d, max_batch=2) as plan:
        x = torch.zeros((B, n, n), device=dev)
        api.mbir_solve(plan, b, w, x, 1, step, prior)
        xs = np64(x)
    wb = np64(w) * np64(b)
    rng = np.random.default_rng(2896)
    for k in range(B):
        pix = rng.integers(0, n * n, 1024)
        ref = step * oracle.radon_adj_at(wb[k], n, pix)
        assert rel(xs[k].ravel()[pix], ref) <= 2e-5


def test_headline_prior_matches_oracle(api):
    """The 26-neighbour prior gradient and value on three 2048^2 slices (tiles
    inside the volume and at its border, at the full side) against the
    oracle: relative L2 1e-5, value 1e-5."""
    n, B = 2048, 3
    f = np.stack([synth.rasterize(n, synth.random_ellipses(n, synth.BASE_SEED + 90 + k, scale=1.0 / n))
                  for k in range(B)])
    f += synth.uniform_field(f.shape, 91, 0.0, 2e-4).astype(np.float64)
    f = f.astype(np.float32).astype(np.float64)
    prior = api.Prior(lam=1e-2, dims=3)
    with api.Plan(n, 8, 2896, max_batch=B) as plan:
        z = torch.zeros((B, 8, 2896), device="cuda:0")
        g, obj = api.mbir_grad(plan, t32(f), z, z, prior)
    Hv, gh = oracle.prior_value_grad(f, 3, **oracle.PAPER_PRIOR)
    assert rel(np64(g), prior.lam * gh) <= 1e-5
    assert abs(float(obj[1]) - prior.lam * Hv) <= 1e-5 * prior.lam * Hv


def test_restart_dots_on_the_full_volume_match_fp64(api):
    """The restart test's inner products <g, z - x> and <g, g> on the whole
    2048^2 x 1024 volume (128 angles, 2896 bins, Poisson weights, 26-neighbour
    prior), against an FP64 reduction of the same FP32 vectors: the gradient
    g = grad Phi(z_k) recomputed by mbir_grad (the same kernels, bit for bit),
    z_k and x_k saved before the iteration.  Bound: 1e-10 of the sum of the
    terms' magnitudes (an FP64 reduction's own error is of that order)."""
    dev = torch.device("cuda:0")
    B = 1024
    n, a, d, b, w = _headline_inputs(B, dev)
    prior = api.Prior(lam=1e-2, dims=3)
    with api.Plan(n, a, d, max_batch=64) as plan:
        x = torch.zeros((B, n, n), device=dev)
        st = api.mbir_solve(plan, b, w, x, 2, 3.75e-6, prior)   # from iteration 2 on, z != x
        xk, zk = x.clone(), st.z.clone()
        api.mbir_solve(plan, b, w, x, 1, 3.75e-6, prior, state=st)
        g, _ = api.mbir_grad(plan, zk, b, w, prior)
        gzx = gg = mag = 0.0
        for s0 in range(0, B, 64):
            gd = g[s0:s0 + 64].double()
            t = gd * (zk[s0:s0 + 64].double() - xk[s0:s0 + 64].double())
            gzx += float(t.sum())
            mag += float(t.abs().sum())
            gg += float((gd * gd).sum())
            del gd, t
    assert abs(st.dots[1] - gg) <= 1e-10 * gg, (st.dots[1], gg)
    assert abs(st.dots[0] - gzx) <= 1e-10 * mag, (st.dots[0], gzx, mag)


# ------------------------------------------------ checkpoints and failures ----
def test_checkpoint_on_storage_resumes_bitwise(api, tmp_path):
    """10 iterations, checkpoint to a file (JSON header + raw x and z), load
    into fresh buffers and a fresh state, 10 more: bit for bit the
    uninterrupted 20-iteration solve (derived step, 3D prior, weights)."""
    B = 3
    _, b = _data(B)
    w = np.random.default_rng(12).uniform(0.4, 1.0, b.shape)
    prior = api.Prior(lam=1e-3, dims=3)
    path = str(tmp_path / "solve.ckpt")
    with api.Plan(N, A, D, max_batch=2) as plan:
        bt, wt = t32(b), t32(w)
        x1 = torch.zeros((B, N, N), device="cuda:0")
        s1 = api.mbir_solve(plan, bt, wt, x1, 20, None, prior)
        x2 = torch.zeros((B, N, N), device="cuda:0")
        s2 = api.mbir_solve(plan, bt, wt, x2, 10, None, prior)
        api.checkpoint_save(path, plan, x2, s2)
        del x2, s2
        x3 = torch.full((B, N, N), 7.0, device="cuda:0")
        s3 = api.checkpoint_load(path, plan, x3)
        assert s3.k == 10 and s3.step == s1.step
        api.mbir_solve(plan, bt, wt, x3, 10, None, prior, state=s3)
        with open(path, "rb") as fh:
            head = fh.readline().decode()
        with pytest.raises(api.TcError):   # geometry mismatch: rejected before any copy
            with api.Plan(64, A, D) as other:
                api.checkpoint_load(path, other, torch.zeros((B, 64, 64), device="cuda:0"))
    assert s3.k == 20 and s3.n_restarts == s1.n_restarts
    assert torch.equal(x3, x1)
    assert torch.equal(s3.z, s1.z)
    assert '"format": "tc-mbir-checkpoint"' in head and f'"k": 10' in head


@pytest.mark.parametrize("after", [0, 2, 7])
def test_injected_copy_failure_is_reported_and_the_plan_stays_usable(api, after):
    """A host-to-device or device-to-host copy of the host-streamed solve that
    fails (injected on the host: the copy is not issued and reports an error)
    gives TC_ERR_CUDA after the copies in flight finish; the next solve on the
    same plan runs normally and matches the resident solve bit for bit.
    Five slices in slabs of two: copies 0..8 are inbound (b, w, x per slab),
    the rest return x slab by slab."""
    B = 5
    _, b = _data(B)
    w = np.random.default_rng(13).uniform(0.5, 1.0, b.shape)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=3)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        api.mbir_solve(plan, t32(b), t32(w), x, 3, step, prior)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        wh = torch.tensor(w, dtype=torch.float32).pin_memory()
        xh = torch.zeros((B, N, N), dtype=torch.float32).pin_memory()
        api.fail_copy_after(after)
        try:
            with pytest.raises(api.TcError) as e:
                api.mbir_solve_host(plan, bh, wh, xh, 3, step, prior)
        finally:
            api.fail_copy_after(-1)
        assert e.value.code == -3 and "injected" in str(e.value)
        xh.zero_()
        api.mbir_solve_host(plan, bh, wh, xh, 3, step, prior)
    assert torch.equal(xh, x.cpu())


def test_plan_that_cannot_fit_returns_oom_and_frees_everything(api):
    """Scratch for 60000 slices of 2048^2 cannot be allocated: tc_plan_create
    returns TC_ERR_OOM and the tables it had already uploaded are released."""
    with api.Plan(2048, 128, 2896, max_batch=1):
        pass   # kernel attributes and the context's lazy state set up once
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(api.TcError) as e:
        api.Plan(2048, 128, 2896, max_batch=60000)
    assert e.value.code == -2
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (2 << 20)


def test_host_solve_argument_checks(api):
    """NULL host buffers are rejected by the C ABI before any copy; the
    binding rejects mis-sized host tensors."""
    L = api.load()
    import ctypes
    with api.Plan(N, A, D) as plan:
        x = torch.zeros((1, N, N), device="cuda:0")
        st = api.SolveState(x)
        cs = st._c()
        opts = api._SolveOpts(2, 1e-4, 1, 0, 0)
        db = torch.zeros((1, A, D), device="cuda:0")
        rc = L.mbir_solve_host(plan.handle, None, None, None, api._ptr(db), None, api._ptr(x), 1, None,
                               ctypes.byref(opts), ctypes.byref(cs), None)
        assert rc == -1
        with pytest.raises(ValueError):
            api.mbir_solve_host(plan, torch.zeros((1, A, D - 2)), None, torch.zeros((1, N, N)), 2, 1e-4)
