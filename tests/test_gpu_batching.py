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


# image sides 64..256 with mixed-radix and Bluestein detector lengths, angle
# counts odd and even, one geometry with arbitrary angles and an axis offset
GROUP_GEOMS = [dict(n=256, n_angles=48, n_det=362), dict(n=64, n_angles=33, n_det=92),
               dict(n=128, n_angles=90, n_det=184), dict(n=32, n_angles=7, n_det=48, center_offset=1.5,
                                                          angles=[0.1, 0.5, 1.1, 1.9, 2.4, 3.0, 3.9])]
GROUP_COUNTS = [3, 5, 2, 4]


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def test_plan_group_matches_per_geometry_plans(api):
    """Work-list launches over the group's items (one per stage and
    geometry class): A, A^T, and the MBIR gradient with weights and the
    26-neighbour prior (objective terms included) agree with one plan per
    geometry to FP32 rounding (the grouped kernels are compiled apart from
    the per-plan ones, so a multiply-add may be fused differently; 1e-6
    relative per geometry and for the objective terms), and a CUDA-graph replay of the
    group equals its eager run bit for bit."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(9)
    with api.PlanGroup(GROUP_GEOMS, GROUP_COUNTS, device=dev) as grp:
        x = torch.tensor(rng.standard_normal(grp.image_numel), dtype=torch.float32, device=dev)
        y = torch.tensor(rng.standard_normal(grp.sino_numel), dtype=torch.float32, device=dev)
        w = torch.tensor(rng.uniform(0.3, 1.0, grp.sino_numel), dtype=torch.float32, device=dev)
        prior = api.Prior(lam=2e-3, dims=3)
        yg = api.radon_fwd_group(grp, x)
        xg = api.radon_adj_group(grp, y)
        gg, og = api.mbir_grad_group(grp, x, y, w, prior)
        torch.cuda.synchronize()
        ref_y, ref_x, ref_g, ref_o = [], [], [], []
        for gm, c, xs, ys, ws in zip(GROUP_GEOMS, GROUP_COUNTS, grp.split_images(x), grp.split_sinos(y),
                                     grp.split_sinos(w)):
            kw = {k: v for k, v in gm.items() if k not in ("n", "n_angles", "n_det")}
            if "angles" in kw:
                kw["angles"] = np.array(kw["angles"])
            with api.Plan(gm["n"], gm["n_angles"], gm["n_det"], max_batch=c, **kw) as p:
                ref_y.append(api.radon_fwd(p, xs.contiguous()).flatten())
                ref_x.append(api.radon_adj(p, ys.contiguous()).flatten())
                g1, o1 = api.mbir_grad(p, xs.contiguous(), ys.contiguous(), ws.contiguous(), prior)
                ref_g.append(g1.flatten())
                ref_o.append(o1)
                torch.cuda.synchronize()
        for got, ref, split in ((yg, ref_y, grp.split_sinos), (xg, ref_x, grp.split_images),
                                (gg, ref_g, grp.split_images)):
            for part_got, part_ref in zip(split(got), ref):
                assert _rel(part_got.flatten(), part_ref) <= 1e-6
        ref_o = torch.stack(ref_o)
        assert float(((og - ref_o).abs() / ref_o.abs()).max()) <= 1e-6
        # the same work captured once and replayed
        yo, xo, go = torch.empty_like(yg), torch.empty_like(xg), torch.empty_like(gg)
        oo = torch.zeros_like(og)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            api.radon_fwd_group(grp, x, yo)
            api.radon_adj_group(grp, y, xo)
            api.mbir_grad_group(grp, x, y, w, prior, grad=go, obj=oo)
        for _ in range(2):
            yo.zero_(), xo.zero_(), go.zero_(), oo.zero_()
            graph.replay()
            torch.cuda.synchronize()
            assert torch.equal(yo, yg) and torch.equal(xo, xg) and torch.equal(go, gg) and torch.equal(oo, og)


def test_plan_group_rejects_bad_arguments(api):
    with pytest.raises(api.TcError):
        api.PlanGroup([(64, 10, 92)], [0])
    with pytest.raises(api.TcError):
        api.PlanGroup([(64, 10, 92), (48, 10, 92)], [1, 1])   # side not a power of two
    with api.PlanGroup([(64, 10, 92)], [2]) as grp:
        with pytest.raises(ValueError):
            api.radon_fwd_group(grp, torch.zeros(grp.image_numel + 1, device="cuda:0"))


def test_spread_chunk_is_a_plan_choice_and_autotuned(api):
    """The spreading chunk (entries staged per pass over a grid row) changes
    only the grouping of each cell's FP32 sum: A^T stays within 1e-6 of the
    default and of the oracle-checked operator, each chunk size is
    bit-reproducible, and the autotuner keeps one of the sizes."""
    dev = torch.device("cuda:0")
    n, a, d, b = 256, 64, 362, 4
    rng = np.random.default_rng(6)
    y = torch.tensor(rng.standard_normal((b, a, d)), dtype=torch.float32, device=dev)
    with api.Plan(n, a, d, max_batch=b) as p:
        assert p.spread_chunk == 1024
        ref = api.radon_adj(p, y).clone()
        for ch in (256, 512, 1024):
            p.spread_chunk = ch
            x1 = api.radon_adj(p, y).clone()
            assert torch.equal(api.radon_adj(p, y), x1)
            assert float((x1 - ref).norm() / ref.norm()) <= 1e-6
        with pytest.raises(api.TcError):
            p.spread_chunk = 300
        best = p.autotune_spread(reps=1)
        assert best in (256, 512, 1024) and p.spread_chunk == best
