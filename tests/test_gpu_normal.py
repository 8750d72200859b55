"""Parity of the normal operator A^T A (Toeplitz-plus-Hankel embedding,
radon_normal) and of the normal-operator MBIR solve with the FP64 oracle,
through the C ABI.

Tolerances: A^T A x within 2e-5 of max |A^T A x| at every pixel (the embedding
is exact; what remains is FP32 rounding of the FFT passes, ~1e-6).  At the
full-size geometries, where the oracle cannot form A^T A x, the embedding is
checked against the gridded radon_adj(radon_fwd(x)) (each within ~2e-6 of
exact) and against the identities <x, A^T A x> = ||A x||^2 and
<y, A^T A x> = <A^T A y, x>.  Solves: <= 1e-3 relative L2 to the oracle after 20
iterations, as for the gridded solver.
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


CASES = [
    # the small configuration: 128^2, 90 angles, 184 bins; three slices in chunks of two
    dict(N=128, A=90, D=184, delta=0.0, B=3, mb=2, theta=None),
    # rotation-axis offset and angles outside [0, pi) (the Hankel term sees them as given)
    dict(N=64, A=20, D=92, delta=0.37, B=2, mb=2, theta="wide"),
    # smallest side, negative offset
    dict(N=16, A=7, D=24, delta=-1.25, B=1, mb=1, theta=None),
    # one angle and a 4-bin detector: the kernels wrap around the detector many
    # times, and the plan's own grid rows are fewer than the N + 1 used here
    dict(N=32, A=1, D=4, delta=0.0, B=2, mb=2, theta=None),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c['N']}_A{c['A']}_D{c['D']}_d{c['delta']}")
def test_normal_matches_oracle(api, case):
    N, A, D, B = case["N"], case["A"], case["D"], case["B"]
    rng = np.random.default_rng(N + A)
    th = None
    if case["theta"] == "wide":
        th = rng.uniform(-1.0, 7.0, A)
    f = np.stack([synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + k)) for k in range(B)])
    f = (f + 0.1 * rng.standard_normal(f.shape)).astype(np.float32).astype(np.float64)
    ref = oracle.normal_op(f, A, D, th, case["delta"])
    with api.Plan(N, A, D, angles=th, max_batch=case["mb"], center_offset=case["delta"]) as plan:
        got = np64(api.radon_normal(plan, t32(f)))
    err = np.max(np.abs(got - ref))
    assert err <= 2e-5 * np.max(np.abs(ref)), err / np.max(np.abs(ref))


def test_normal_in_place_and_prepared_equal(api):
    N, A, D = 64, 30, 92
    f = synth.random_start((3, N, N), 5).astype(np.float32)
    with api.Plan(N, A, D, max_batch=2) as plan:
        plan.prepare_normal()
        x = t32(f)
        out = api.radon_normal(plan, x)
        api.radon_normal(plan, x, out=x)
        torch.cuda.synchronize()
    assert torch.equal(out, x)


@pytest.mark.parametrize("geom", [(2048, 128, 2896), (1024, 360, 1448)], ids=["2048_128_2896", "1024_360_1448"])
def test_normal_full_size_against_gridded_and_identities(api, geom):
    """The benchmark geometries: 2048^2 with 128 angles and 2896 bins, and
    1024^2 with 360 angles and 1448 bins, two slices per launch."""
    N, A, D = geom
    x = torch.tensor(synth.phantom_slices(N, 2)[0], dtype=torch.float32, device="cuda:0")
    y = torch.tensor(synth.random_start((2, N, N), 11), dtype=torch.float32, device="cuda:0")
    with api.Plan(N, A, D, max_batch=2) as plan:
        nx = api.radon_normal(plan, x)
        ny = api.radon_normal(plan, y)
        ax = api.radon_fwd(plan, x)
        ay = api.radon_fwd(plan, y)
        gx = api.radon_adj(plan, ax)
        torch.cuda.synchronize()
    nx, ny, ax, ay, gx = (np64(t) for t in (nx, ny, ax, ay, gx))
    xd, yd = np64(x), np64(y)
    assert rel(nx, gx) <= 2e-5
    e = float(np.sum(ax * ax))
    assert abs(float(np.sum(xd * nx)) - e) <= 1e-5 * e
    s = float(np.linalg.norm(ax) * np.linalg.norm(ay))
    assert abs(float(np.sum(yd * nx)) - float(np.sum(xd * ny))) <= 1e-5 * s
    assert abs(float(np.sum(yd * nx)) - float(np.sum(ay * ax))) <= 2e-5 * s


N, A, D = 128, 90, 184


def _data(B):
    ells = [synth.random_ellipses(N, synth.BASE_SEED + k) for k in range(B)]
    b = np.stack([synth.ellipse_line_integrals(e, oracle.default_angles(A), D) for e in ells])
    return b.astype(np.float32).astype(np.float64)


def _step(lam):
    v0 = synth.random_start((1, N, N), 7)
    L = 1.05 * oracle.power_norm(N, A, D, None, v0, 30)
    return 1.0 / (L + 8.0 * lam / ((1 / 0.7) ** 2 * 1e-4))


@pytest.mark.parametrize("dims", [2, 3])
def test_normal_solve_matches_oracle_and_gridded(api, dims):
    B = 2
    b = _data(B)
    lam = 1e-3
    step = _step(lam)
    prior = api.Prior(lam=lam, dims=dims)
    xo, log = oracle.mbir_solve(b, None, N, 20, step, lam=lam,
                                prior=dict(p=prior.p, sigma=prior.sigma, c=prior.c),
                                dims=dims, return_log=True)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), None, x, 20, step, prior, normal=True)
        xg = torch.zeros((B, N, N), device="cuda:0")
        sg = api.mbir_solve(plan, t32(b), None, xg, 20, step, prior)
    assert st.k == 20
    assert st.n_restarts == sum(e["restart"] for e in log)
    assert rel(np64(x), xo) <= 1e-3
    assert rel(np64(x), np64(xg)) <= 1e-4
    # data term at the last gradient point, through 1/2 <z, A^T A z> - <z, A^T b> + 1/2 ||b||^2:
    # the operator's FP32 rounding (2e-6) acts on 1/2 <z, A^T A z> ~ 1/2 ||b||^2, not on the residual
    assert abs(st.obj[0] - sg.obj[0]) <= 2e-6 * 0.5 * float(np.sum(b * b))
    assert abs(st.obj[1] - sg.obj[1]) <= 1e-4 * sg.obj[1]


@pytest.mark.parametrize("restart", [True, False])
def test_normal_solve_without_prior(api, restart):
    """No prior: the solver takes the separate restart-dot and update kernels."""
    B = 2
    b = _data(B)
    step = _step(0.0)
    xo, log = oracle.mbir_solve(b, None, N, 15, step, lam=0.0, dims=2, restart=restart, return_log=True)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        st = api.mbir_solve(plan, t32(b), None, x, 15, step, None, restart=restart, normal=True)
        xg = torch.zeros((B, N, N), device="cuda:0")
        sg = api.mbir_solve(plan, t32(b), None, xg, 15, step, None, restart=restart)
    assert st.k == 15 and st.obj[1] == 0.0
    assert st.n_restarts == sum(e["restart"] for e in log)
    assert rel(np64(x), xo) <= 1e-3
    assert rel(np64(x), np64(xg)) <= 1e-4
    assert abs(st.obj[0] - sg.obj[0]) <= 2e-6 * 0.5 * float(np.sum(b * b))


def test_normal_solve_resume_equals_uninterrupted_bitwise(api):
    b = _data(2)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=2)
    with api.Plan(N, A, D, max_batch=2) as plan:
        bt = t32(b)
        x1 = torch.zeros((2, N, N), device="cuda:0")
        api.mbir_solve(plan, bt, None, x1, 12, step, prior, normal=True)
        x2 = torch.zeros((2, N, N), device="cuda:0")
        st = api.mbir_solve(plan, bt, None, x2, 5, step, prior, normal=True)
        api.mbir_solve(plan, bt, None, x2, 7, step, prior, state=st, normal=True)
    assert st.k == 12
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("n_iter", [4, 1])
def test_normal_host_streamed_solve_matches_device_solve(api, n_iter):
    """Five slices in slabs of two: A^T b of slab c is formed as soon as slab c
    is resident; the last iteration returns x slab by slab."""
    B = 5
    b = _data(B)
    step = _step(1e-3)
    prior = api.Prior(lam=1e-3, dims=3)
    with api.Plan(N, A, D, max_batch=2) as plan:
        x = torch.zeros((B, N, N), device="cuda:0")
        sd = api.mbir_solve(plan, t32(b), None, x, n_iter, step, prior, normal=True)
        bh = torch.tensor(b, dtype=torch.float32).pin_memory()
        xh = torch.zeros((B, N, N), dtype=torch.float32).pin_memory()
        sh = api.mbir_solve_host(plan, bh, None, xh, n_iter, step, prior, normal=True)
    assert torch.equal(xh, x.cpu())
    assert sh.k == sd.k == n_iter and sh.n_restarts == sd.n_restarts
    assert torch.equal(sh.z.cpu(), sd.z.cpu())
    assert abs(sh.obj[0] - sd.obj[0]) <= 1e-12 * abs(sd.obj[0])


def test_normal_solve_rejections(api):
    b = _data(1)
    w = np.ones_like(b)
    with api.Plan(N, A, D) as plan:
        x = torch.zeros((1, N, N), device="cuda:0")
        with pytest.raises(api.TcError) as e:
            api.mbir_solve(plan, t32(b), t32(w), x, 2, 1e-3, None, normal=True)
        assert e.value.code == -1
        with pytest.raises(api.TcError) as e:
            api.mbir_solve(plan, t32(b), None, x, 2, 1e-3, None, restart="monotone", normal=True)
        assert e.value.code == -1


def test_normal_largest_side_against_gridded(api):
    """N = 4096, the largest side: the only size whose table build runs the
    FP64 FFT at G = 8192 (128 KB of shared memory a CTA) and whose row pass
    runs k_nrm_row<12>.  Few angles (A = 8, D = 5792) keep the gridded check
    A^T (A x) affordable; the two agree within 2e-5 relative L2."""
    n, a, d = 4096, 8, 5792
    x = torch.tensor(synth.uniform_field((1, n, n), 4096), device="cuda:0")
    with api.Plan(n, a, d, max_batch=1) as plan:
        nx = api.radon_normal(plan, x)
        gx = api.radon_adj(plan, api.radon_fwd(plan, x))
        torch.cuda.synchronize()
        assert float((nx - gx).norm() / gx.norm()) <= 2e-5


def test_unprepared_normal_inside_a_capture_is_refused(api):
    """The first normal-operator call builds tables (allocation, synchronisation),
    which a CUDA-graph capture cannot record: inside a capture the unprepared
    call returns TC_ERR_UNSUPPORTED without touching the stream; once prepared,
    the captured call replays and matches the eager result."""
    n, a, d = 64, 30, 92
    x = torch.tensor(synth.uniform_field((2, n, n), 64), device="cuda:0")
    out = torch.empty_like(x)
    with api.Plan(n, a, d, max_batch=2) as plan:
        api.radon_fwd(plan, x)   # kernels loaded before any capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        codes = []
        with torch.cuda.graph(g):
            try:
                api.radon_normal(plan, x, out=out)
            except api.TcError as e:
                codes.append(e.code)
        assert codes == [-5]
        plan.prepare_normal()
        eager = api.radon_normal(plan, x).clone()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2):
            api.radon_normal(plan, x, out=out)
        out.zero_()
        g2.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
