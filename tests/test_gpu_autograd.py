"""Autograd through radon_fwd: the backward is the hand-written A^T kernel.

Loss = 1/2 sum W (A x - b)^2 + lam H(x) (the prior through mbir_grad's
path is not autograd; here the prior term is added from the library's own
gradient so the test checks the radon_fwd backward).  Checked by central
finite differences (step 1e-3) on 32 seeded directions, with the loss
accumulated in FP64, and against the FP64 oracle gradient.
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


def test_backward_matches_finite_differences_and_oracle(api):
    N, A, D, B = 64, 48, 92, 2
    rng = np.random.default_rng(31)
    x0 = np.stack([synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED + k)) for k in range(B)])
    b = rng.standard_normal((B, A, D))
    w = rng.uniform(0.2, 1.0, (B, A, D))
    dev = torch.device("cuda:0")
    bt = torch.tensor(b, dtype=torch.float32, device=dev)
    wt = torch.tensor(w, dtype=torch.float32, device=dev)
    with api.Plan(N, A, D, max_batch=B) as plan:
        def loss(xt):
            y = api.radon(xt, plan)
            r = (y - bt).double()
            return 0.5 * (wt.double() * r * r).sum()

        x = torch.tensor(x0, dtype=torch.float32, device=dev, requires_grad=True)
        L = loss(x)
        L.backward()
        g = x.grad.double()
        h = 1e-3
        dirs = torch.tensor(rng.standard_normal((32, B, N, N)), dtype=torch.float32, device=dev)
        with torch.no_grad():
            for d in dirs:
                d = d / d.norm()
                fd = (loss(x + h * d) - loss(x - h * d)) / (2 * h)
                an = (g * d.double()).sum()
                assert abs(float(fd - an)) <= 1e-3 * float(g.norm()), (float(fd), float(an))
    xo = x0.astype(np.float32).astype(np.float64)
    _, go = oracle.data_grad(xo, b.astype(np.float32).astype(np.float64),
                             w.astype(np.float32).astype(np.float64))
    assert float(np.linalg.norm(g.cpu().numpy() - go) / np.linalg.norm(go)) <= 1e-4


def test_backward_at_the_differentiation_workload_size(api):
    """One slice of the differentiation workload: 1024^2, 360 angles, 1448
    bins.  The radon_fwd backward (the A^T kernel) against central finite
    differences (step 1e-3) on 32 seeded directions, and the gradient of
    1/2 sum W (A x - b)^2 against the FP64 oracle at 512 sampled pixels stored
    by tests/golden/make_oracle_golden.py (relative L2 over the sample <= 1e-4,
    as above), with the loss itself within 1e-5.

    The stored inputs are scaled by s = 2^-10 (exact in floating point), and
    the stored loss and gradient by s^2 and s: the loss is quadratic in (x, b)
    jointly.  At the stored scale the FP32 forward's rounding, about 1e-6 of
    the loss, would swamp a 1e-3 finite-difference step; it shrinks with the
    residual, the directional derivative only with its square root."""
    import make_oracle_golden as mk
    c = mk.AUTOGRAD
    N, A, D = c["N"], c["A"], c["D"]
    ref = np.load(mk.autograd_path())
    x0, b, w = mk.autograd_inputs()
    s = np.float32(2.0 ** -10)
    x0, b = x0 * s, b * s
    ref = dict(pix=ref["pix"], g=ref["g"] * float(s), loss=float(ref["loss"]) * float(s) ** 2)
    dev = torch.device("cuda:0")
    bt = torch.tensor(b[None], device=dev)
    wt = torch.tensor(w[None], device=dev)
    with api.Plan(N, A, D, max_batch=1) as plan:
        def loss(xt):
            y = api.radon(xt, plan)
            r = (y - bt).double()
            return 0.5 * (wt.double() * r * r).sum()

        x = torch.tensor(x0[None], device=dev, requires_grad=True)
        L = loss(x)
        L.backward()
        g = x.grad.double()
        assert abs(float(L.detach()) - ref["loss"]) <= 1e-5 * ref["loss"]
        gs = g[0].flatten()[torch.as_tensor(ref["pix"], dtype=torch.long, device=dev)].cpu().numpy()
        err = float(np.linalg.norm(gs - ref["g"]) / np.linalg.norm(ref["g"]))
        assert err <= 1e-4, err
        rng = np.random.default_rng(1448)
        h = 1e-3
        gn = float(g.norm())
        with torch.no_grad():
            for _ in range(32):
                d = torch.tensor(rng.standard_normal((1, N, N)), dtype=torch.float32, device=dev)
                d = d / d.norm()
                fd = (loss(x + h * d) - loss(x - h * d)) / (2 * h)
                an = (g * d.double()).sum()
                assert abs(float(fd - an)) <= 1e-3 * gn, (float(fd), float(an))
