"""The allocation-free prior entry point, tc_prior_grad_noalloc.

It serves callers that cannot call cudaMalloc (a framework whose caching
allocator owns the device memory, or a loop that must not risk an
allocation's implicit device synchronisation) and so cannot create a plan.
Its scratch is a fixed device array inside the library, shared by all calls.
This test calls it through the C ABI twice in a row, on different inputs, and
compares each result with the plan-based mbir_grad (zero data weights leave
only the prior), within the tolerance of the other prior tests.  The file
name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_12934_gb300 import api as a
    L = a.load()
    L.tc_prior_grad_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(a._Prior),
                                        ctypes.c_void_p, ctypes.c_void_p]
    L.tc_prior_grad_noalloc.restype = ctypes.c_int
    return a


@pytest.mark.parametrize("dims", [3, 2])
def test_noalloc_prior_matches_plan_path_on_two_calls(api, dims):
    L = api.load()
    N, A, D, B = 128, 30, 184, 3
    prior = api.Prior(lam=0.5, dims=dims)
    stream = torch.cuda.current_stream()
    with api.Plan(N, A, D, max_batch=2) as plan:
        b = torch.zeros((B, A, D), device="cuda:0")
        wzero = torch.zeros((B, A, D), device="cuda:0")
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            x = torch.tensor(rng.uniform(0, 1, (B, N, N)), dtype=torch.float32, device="cuda:0")
            g_ref, obj = api.mbir_grad(plan, x, b, wzero, prior)
            g = torch.zeros_like(x)
            h = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
            pc = prior._c()
            rc = L.tc_prior_grad_noalloc(x.data_ptr(), g.data_ptr(), N, B, ctypes.byref(pc),
                                         h.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            torch.cuda.synchronize()
            assert rc == 0
            assert float((g - g_ref).norm() / g_ref.norm()) <= TOL
            href = float(obj[1])
            assert abs(float(h[0]) - href) <= TOL * abs(href)


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    L = api.load()
    pc = api.Prior(dims=3)._c()
    x = torch.zeros((1, 16, 16), device="cuda:0")
    g = torch.zeros_like(x)
    rc = L.tc_prior_grad_noalloc(x.data_ptr(), g.data_ptr(), 8192, 1, ctypes.byref(pc), None, None)
    assert rc == -1


def test_noalloc_rejects_overlapping_input_and_output(api):
    """grad is written at one slice while other blocks still read x above and
    below it, so x and grad must not overlap (in place or shifted)."""
    L = api.load()
    pc = api.Prior(dims=3)._c()
    v = torch.zeros((4, 16, 16), device="cuda:0")
    for xo, go in ((0, 0), (0, 1), (1, 0)):
        rc = L.tc_prior_grad_noalloc(v[xo].data_ptr(), v[go].data_ptr(), 16, 3, ctypes.byref(pc), None, None)
        assert rc == -1


@pytest.mark.parametrize("n,batch", [(100, 5), (3, 4)])
@pytest.mark.parametrize("dims", [2, 3])
def test_noalloc_at_sides_the_plans_never_use(api, n, batch, dims):
    """Sides that are not powers of two, smaller than a prior tile or not a
    multiple of it (only border tiles, masked pairs) against the FP64 oracle's
    qGGMRF value and gradient, on two calls in a row."""
    import oracle
    L = api.load()
    prior = api.Prior(lam=0.5, dims=dims)
    stream = torch.cuda.current_stream()
    pd = dict(p=prior.p, sigma=prior.sigma, c=prior.c)
    for call in range(2):
        rng = np.random.default_rng(7 * n + call)
        f = rng.uniform(0, 1, (batch, n, n)).astype(np.float32)
        x = torch.tensor(f, device="cuda:0")
        g = torch.zeros_like(x)
        h = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
        pc = prior._c()
        rc = L.tc_prior_grad_noalloc(x.data_ptr(), g.data_ptr(), n, batch, ctypes.byref(pc),
                                     h.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert rc == 0
        Hv, gh = oracle.prior_value_grad(f.astype(np.float64), dims, **pd)
        gd = g.double().cpu().numpy()
        assert float(np.linalg.norm(gd - prior.lam * gh) / np.linalg.norm(prior.lam * gh)) <= TOL
        assert abs(float(h[0]) - prior.lam * Hv) <= TOL * prior.lam * Hv


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_prior_at_the_ends_of_the_exponent_range(api, p):
    """p = 1 and p = 2 (q = 2 - p = 1 and 0), on a piecewise-constant volume
    whose neighbour differences are often exactly zero: at q = 0 the kernel's
    |d|^q must still be 1 there (a zero difference gives a zero pair value,
    not 0 * inf).  Against the FP64 oracle, 3D and 2D."""
    import oracle
    L = api.load()
    stream = torch.cuda.current_stream()
    n, batch = 64, 6
    rng = np.random.default_rng(int(p * 10) + 1)
    f = (np.round(rng.uniform(0, 1, (batch, n, n)) * 3) / 3).astype(np.float32)
    for dims in (3, 2):
        prior = api.Prior(p=p, lam=0.5, dims=dims)
        x = torch.tensor(f, device="cuda:0")
        g = torch.zeros_like(x)
        h = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
        pc = prior._c()
        rc = L.tc_prior_grad_noalloc(x.data_ptr(), g.data_ptr(), n, batch, ctypes.byref(pc),
                                     h.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert rc == 0
        Hv, gh = oracle.prior_value_grad(f.astype(np.float64), dims, p=p, sigma=prior.sigma, c=prior.c)
        gd = g.double().cpu().numpy()
        assert np.isfinite(gd).all() and np.isfinite(float(h[0]))
        assert float(np.linalg.norm(gd - prior.lam * gh) / np.linalg.norm(prior.lam * gh)) <= TOL, (p, dims)
        assert abs(float(h[0]) - prior.lam * Hv) <= TOL * prior.lam * Hv, (p, dims)
