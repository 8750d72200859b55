"""Parity of the CUDA NUFFT Radon operators with the FP64 oracle (C ABI).

Tolerances (element-wise on the same seeded inputs):
  * A and A^T: relative L2 <= 2e-5 against the exact NUDFT oracle (the ES
    kernel at w = 7, sigma = 2 has ~1e-6 relative error; FP32 FFTs add ~1e-6);
  * adjoint mismatch of the GPU pair |<Ax,y> - <x,A^T y>| / (|Ax||y|) <= 1e-5;
  * sampled entries at full size: max error <= 2e-5 of the output's RMS.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_12934_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 2e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_12934_gb300 import api as a
    a.load()
    return a


def dev():
    return torch.device("cuda", 0)


def t32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


GEOMS = [
    # (N, A, D, angles)  -- config-1 size first
    (128, 90, 184, None),
    (16, 7, 24, "random"),
    (32, 20, 46, "random2pi"),
    (64, 33, 92, None),
    (256, 64, 362, None),
    (64, 1, 92, None),
    (32, 13, 128, "random"),
]


def _angles(kind, A, seed):
    if kind is None:
        return None
    rng = np.random.default_rng(seed)
    hi = math.pi if kind == "random" else 2 * math.pi
    return rng.uniform(-0.3, hi, A)


@pytest.mark.parametrize("N,A,D,kind", GEOMS)
def test_forward_and_adjoint_match_oracle(api, N, A, D, kind):
    th = _angles(kind, A, N + A)
    rng = np.random.default_rng(N * 7 + A)
    B = 2
    f = np.stack([synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + k)) for k in range(B)])
    f[1] += 0.1 * rng.standard_normal((N, N))
    yy = rng.standard_normal((B, A, D))
    with api.Plan(N, A, D, angles=th, max_batch=2) as plan:
        y = api.radon_fwd(plan, t32(f)).double().cpu().numpy()
        x = api.radon_adj(plan, t32(yy)).double().cpu().numpy()
    thv = th if th is not None else oracle.default_angles(A)
    # the oracle sees exactly the float32 inputs the GPU saw
    f32 = f.astype(np.float32).astype(np.float64)
    y32 = yy.astype(np.float32).astype(np.float64)
    yo = oracle.radon_fwd(f32, A, D, thv)
    xo = oracle.radon_adj(y32, N, thv)
    for k in range(B):
        assert rel(y[k], yo[k]) <= REL_TOL, (k, rel(y[k], yo[k]))
        assert rel(x[k], xo[k]) <= REL_TOL, (k, rel(x[k], xo[k]))


def test_gpu_pair_is_adjoint(api):
    N, A, D = 128, 90, 184
    rng = np.random.default_rng(5)
    x = t32(rng.standard_normal((3, N, N)))
    y = t32(rng.standard_normal((3, A, D)))
    with api.Plan(N, A, D, max_batch=3) as plan:
        Ax = api.radon_fwd(plan, x).double()
        Aty = api.radon_adj(plan, y).double()
    lhs = float((Ax * y.double()).sum())
    rhs = float((x.double() * Aty).sum())
    scale = float(Ax.norm() * y.double().norm())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_chunked_batch_equals_single_slices_bitwise(api):
    N, A, D = 64, 40, 92
    rng = np.random.default_rng(11)
    x = t32(rng.standard_normal((5, N, N)))
    y = t32(rng.standard_normal((5, A, D)))
    with api.Plan(N, A, D, max_batch=2) as p2, api.Plan(N, A, D, max_batch=1) as p1:
        yb = api.radon_fwd(p2, x)
        xb = api.radon_adj(p2, y)
        for k in range(5):
            assert torch.equal(api.radon_fwd(p1, x[k:k + 1].contiguous())[0], yb[k])
            assert torch.equal(api.radon_adj(p1, y[k:k + 1].contiguous())[0], xb[k])


def test_repeat_runs_are_bit_identical(api):
    N, A, D = 128, 90, 184
    rng = np.random.default_rng(3)
    x = t32(rng.standard_normal((2, N, N)))
    y = t32(rng.standard_normal((2, A, D)))
    with api.Plan(N, A, D, max_batch=2) as plan:
        r1 = api.radon_fwd(plan, x).clone()
        s1 = api.radon_adj(plan, y).clone()
        for _ in range(3):
            assert torch.equal(api.radon_fwd(plan, x), r1)
            assert torch.equal(api.radon_adj(plan, y), s1)


def test_empty_batch_and_bad_arguments(api):
    N, A, D = 32, 10, 46
    with api.Plan(N, A, D) as plan:
        z = torch.empty((0, N, N), device=dev())
        out = api.radon_fwd(plan, z)
        assert out.shape == (0, A, D)
        with pytest.raises(ValueError):
            api.radon_fwd(plan, torch.zeros((1, N, N + 1), device=dev()))
        with pytest.raises(ValueError):
            api.radon_fwd(plan, torch.zeros((1, N, N), device=dev(), dtype=torch.float64))
    with pytest.raises(api.TcError):
        api.Plan(48, 10, 46)


def test_theta_zero_gives_column_sums(api):
    """At theta = 0 the operator must reduce to exact column sums (NUFFT error only)."""
    N, D = 64, 92
    rng = np.random.default_rng(8)
    f = rng.uniform(0, 1, (1, N, N))
    with api.Plan(N, 1, D, angles=np.array([0.0])) as plan:
        y = api.radon_fwd(plan, t32(f)).double().cpu().numpy()[0, 0]
    off = (D - N) // 2
    col = f.astype(np.float32).astype(np.float64)[0].sum(axis=0)
    assert np.abs(y[off:off + N] - col).max() <= 2e-5 * np.abs(col).max()


@pytest.mark.parametrize("N,A,D", [(2048, 128, 2896), (512, 180, 724),
                                   (2048, 400, 2048),   # 400 projections x 2048 bins (D = 2^11)
                                   (2048, 202, 2448)])  # 202 projections x 2448 bins (D = 16 * 9 * 17)
def test_full_size_sampled_entries(api, N, A, D):
    """Full-size operators in the batched launch configuration (two slices per
    launch), checked on 1024 entries (angle, bin) drawn over the whole detector
    and 1024 pixels, against the oracle's closed-form values stored by
    tests/golden/make_oracle_golden.py: relative L2 over the sample <= 2e-5."""
    import make_oracle_golden as mk
    ref = np.load(mk.sampled_path(N, A, D))
    f, yy = mk.sampled_inputs(N, A, D)
    rng = np.random.default_rng(N + 1)
    # slice 0 is the stored one; slice 1 only makes the launch a batch
    fb = np.stack([f, rng.random((N, N)).astype(np.float32)])
    yb = np.stack([yy, rng.random((A, D)).astype(np.float32)])
    with api.Plan(N, A, D, max_batch=2) as plan:
        y = api.radon_fwd(plan, t32(fb))[0].double().cpu().numpy()
        x = api.radon_adj(plan, t32(yb))[0].double().cpu().numpy()
    ys = y[ref["ai"], ref["ii"]]
    assert rel(ys, ref["y"]) <= REL_TOL, rel(ys, ref["y"])
    xs = x.ravel()[ref["pix"]]
    assert rel(xs, ref["x"]) <= REL_TOL, rel(xs, ref["x"])


@pytest.mark.parametrize("N,A,D,delta,kind", [
    (64, 33, 92, 3.4, "random2pi"),     # mixed-radix detector DFT, flipped angles
    (128, 90, 184, -11.75, None),       # D = 8 * 23: Bluestein
    (32, 13, 46, 23.0, "random"),       # |delta| = D/2, the largest allowed
])
def test_rotation_axis_offset_matches_oracle(api, N, A, D, delta, kind):
    """Axis offset delta (Sec. 4.1 Fourier shift): forward and adjoint against
    the oracle's shifted operator, and the adjoint identity of the GPU pair."""
    th = _angles(kind, A, N + 5)
    rng = np.random.default_rng(N + D)
    f = synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + 3))[None]
    yy = rng.standard_normal((1, A, D))
    with api.Plan(N, A, D, angles=th, center_offset=delta) as plan:
        y = api.radon_fwd(plan, t32(f)).double().cpu().numpy()
        x = api.radon_adj(plan, t32(yy)).double().cpu().numpy()
    thv = th if th is not None else oracle.default_angles(A)
    f32 = f.astype(np.float32).astype(np.float64)
    y32 = yy.astype(np.float32).astype(np.float64)
    assert rel(y, oracle.radon_fwd(f32, A, D, thv, delta=delta)) <= REL_TOL
    assert rel(x, oracle.radon_adj(y32, N, thv, delta=delta)) <= REL_TOL
    lhs, rhs = float(np.sum(y * y32)), float(np.sum(f32 * x))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(y) * np.linalg.norm(y32)


@pytest.mark.parametrize("delta", [float("nan"), 46.5, -1e9])
def test_rotation_axis_offset_out_of_range_is_rejected(api, delta):
    with pytest.raises(api.TcError):
        api.Plan(32, 8, 92, center_offset=delta)


@pytest.mark.parametrize("N,A,D", [(2048, 128, 2896), (128, 90, 184), (16, 7, 24)])
def test_tma_staged_column_pass_equals_plain_loads(api, N, A, D):
    """With two or more column pairs per CTA the forward column pass stages
    its image strip by TMA; with one it reads global memory directly.  The
    arithmetic is the same, so the outputs agree bit for bit."""
    rng = np.random.default_rng(N + 1)
    x = t32(rng.standard_normal((2, N, N)))
    with api.Plan(N, A, D, max_batch=2) as plan:
        plan.set_launch(2, 2)
        y_tma = api.radon_fwd(plan, x).clone()
        plan.set_launch(2, 1)
        y_plain = api.radon_fwd(plan, x).clone()
        assert load_status(api, plan) == 0
    assert torch.equal(y_tma, y_plain)


def load_status(api, plan):
    return api.load().tc_plan_status(plan.handle)


def test_bounded_wait_times_out_and_the_context_stays_usable(api):
    """A barrier that never completes: the bounded wait expires (2 ms), the
    kernel records TC_ERR_TIMEOUT and returns; later work runs normally."""
    L = api.load()
    assert L.tc_selftest_wait_timeout(None) == -4
    N, A, D = 64, 33, 92
    f = synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + 7))[None]
    with api.Plan(N, A, D) as plan:
        y = api.radon_fwd(plan, t32(f)).double().cpu().numpy()
        assert L.tc_plan_status(plan.handle) == 0
    yo = oracle.radon_fwd(f.astype(np.float32).astype(np.float64), A, D)
    assert rel(y, yo) <= REL_TOL


def test_largest_image_side(api):
    """N = 4096 (the largest side): one column pair per CTA (plain loads) and
    a detector DFT of 5792 = 32 * 181 bins (mixed radix with the radix 181);
    sampled outputs against the oracle's closed form."""
    N, A, D = 4096, 24, 5792
    f = synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + 11)).astype(np.float32)[None]
    rng = np.random.default_rng(4096)
    yy = rng.standard_normal((1, A, D)).astype(np.float32)
    with api.Plan(N, A, D) as plan:
        y = api.radon_fwd(plan, t32(f)).double().cpu().numpy()[0]
        x = api.radon_adj(plan, t32(yy)).double().cpu().numpy()[0]
    ai = rng.integers(0, A, 12)
    ii = rng.integers(D // 4, 3 * D // 4, 12)
    ys = oracle.radon_fwd_at(f[0].astype(np.float64), A, D, ai, ii)
    assert np.abs(y[ai, ii] - ys).max() <= REL_TOL * 2 * float(np.sqrt(np.mean(y ** 2)))
    pix = rng.integers(0, N * N, 12)
    xs = oracle.radon_adj_at(yy[0].astype(np.float64), N, pix)
    assert np.abs(x.ravel()[pix] - xs).max() <= REL_TOL * 2 * float(np.sqrt(np.mean(x ** 2)))


def test_detector_beyond_the_shared_memory_limit_is_unsupported(api):
    with pytest.raises(api.TcError) as e:
        api.Plan(64, 8, 16384)   # mixed radix would need 393 KB of shared memory
    assert e.value.code == -5
