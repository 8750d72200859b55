"""Batching: uneven geometries in one CUDA graph, launch-shape autotuning.

A batch of slices with different sizes and angle counts (one plan per
geometry) is captured into a single CUDA graph and replayed; every output
must equal the eager one-plan-at-a-time result bit for bit, and the plain
one-slice-per-launch form must equal the batched form bit for bit.  The
autotuner may change slices per launch and column pairs per CTA, never the
result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_12934_gb300 import api as a
    a.load()
    return a


GEOMS = [(64, 32, 92, 3), (128, 64, 184, 2), (256, 48, 362, 1), (128, 90, 184, 4)]


def test_uneven_batch_captured_in_one_graph(api):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2)
    plans, xs, ys, eager = [], [], [], []
    for n, a, d, b in GEOMS:
        p = api.Plan(n, a, d, max_batch=b)
        x = torch.tensor(rng.standard_normal((b, n, n)), dtype=torch.float32, device=dev)
        plans.append(p)
        xs.append(x)
        ys.append(torch.empty((b, a, d), device=dev))
        eager.append(api.radon_fwd(p, x).clone())  # also loads the kernels before capture
    adj_in = [torch.tensor(rng.standard_normal(y.shape), dtype=torch.float32, device=dev) for y in ys]
    adj_out = [torch.empty_like(x) for x in xs]
    adj_eager = [api.radon_adj(p, yi).clone() for p, yi in zip(plans, adj_in)]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for p, x, y, yi, xo in zip(plans, xs, ys, adj_in, adj_out):
            api.radon_fwd(p, x, y)
            api.radon_adj(p, yi, xo)
    for _ in range(2):
        for y in ys:
            y.zero_()
        g.replay()
        torch.cuda.synchronize()
        for y, e in zip(ys, eager):
            assert torch.equal(y, e)
        for xo, e in zip(adj_out, adj_eager):
            assert torch.equal(xo, e)
    for p in plans:
        p.close()


def test_plain_one_slice_per_launch_equals_batched(api):
    dev = torch.device("cuda:0")
    n, a, d, b = 128, 90, 184, 6
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.standard_normal((b, n, n)), dtype=torch.float32, device=dev)
    with api.Plan(n, a, d, max_batch=b) as pb, api.Plan(n, a, d, max_batch=1) as p1:
        yb = api.radon_fwd(pb, x)
        y1 = torch.stack([api.radon_fwd(p1, x[k:k + 1].contiguous())[0] for k in range(b)])
    assert torch.equal(yb, y1)


def test_autotune_changes_launch_shape_not_results(api):
    dev = torch.device("cuda:0")
    n, a, d, b = 256, 64, 362, 8
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.standard_normal((b, n, n)), dtype=torch.float32, device=dev)
    y = torch.tensor(rng.standard_normal((b, a, d)), dtype=torch.float32, device=dev)
    with api.Plan(n, a, d, max_batch=b) as p:
        f0, a0 = api.radon_fwd(p, x).clone(), api.radon_adj(p, y).clone()
        chunk, cp = p.autotune(reps=1)
        assert 1 <= chunk <= b and cp in (1, 2, 4)
        assert torch.equal(api.radon_fwd(p, x), f0)
        assert torch.equal(api.radon_adj(p, y), a0)
        for ch, c in ((1, 1), (3, 4), (b, 2)):
            p.set_launch(ch, c)
            assert torch.equal(api.radon_fwd(p, x), f0)
            assert torch.equal(api.radon_adj(p, y), a0)
        with pytest.raises(api.TcError):
            p.set_launch(b + 1, 0)
