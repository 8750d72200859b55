"""Writes the stored expected values of the full-size parity tests.

Every value written here comes from the FP64 oracle (``oracle/``) on inputs
drawn by the seeded generators of ``paper_2304_12934_gb300.synth``; nothing
comes from the CUDA path.  The oracle is too slow to run inside a GPU test at
these sizes (one 1024^2 x 360-angle exact forward takes minutes), so the
tests read the files this script writes.

Fixtures (``tests/golden/*.npz``):

* ``sampled_<N>_<A>_<D>.npz`` -- A and A^T of one slice at the full-size
  geometries, on 1024 entries (angle, bin) drawn over the whole detector and
  1024 pixels, from the Dirichlet closed form (Sec. 2.1 Eq. radon_transform
  through the Fourier-slice theorem, Eq. fourier_radon; Sec. 3 Eq.
  transpose).  Inputs: uniform_field images and sinograms (bit-identical on
  every platform).
* ``noisy_512_180_724.npz`` -- the noisy, weighted solve: one 512^2 slice,
  180 angles, 724 bins, Poisson data at I0 = 1e4 with count weights (Sec. 5:
  b = -log(I/I0)), 8-neighbour qGGMRF (Sec. 3 Eqs. reg2, reg3) with
  lambda = 1e-2, accelerated gradient with gradient restart (Sec. 3, last
  paragraph) for 50 iterations.  The Poisson draw uses libm, so b and w are
  stored with the result.
* ``autograd_1024_360_1448.npz`` -- the gradient of 1/2 sum W (A x - b)^2
  (Sec. 3 Eq. gradient) at 512 sampled pixels for one 1024^2 slice with 360
  angles and 1448 bins; inputs are uniform_field draws.

  python tests/golden/make_oracle_golden.py [sampled|noisy|autograd|all]
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2304_12934_gb300 import synth  # noqa: E402

SAMPLED_GEOMS = [(2048, 128, 2896), (512, 180, 724), (2048, 400, 2048), (2048, 202, 2448)]
N_SAMPLES = 1024


def sampled_inputs(N, A, D):
    """Seeded inputs of the sampled full-size check (shared with the test)."""
    f = synth.uniform_field((N, N), synth.BASE_SEED + N + A)
    yy = synth.uniform_field((A, D), synth.BASE_SEED + D + A, -1.0, 1.0)
    return f, yy


def sampled_path(N, A, D):
    return os.path.join(HERE, f"sampled_{N}_{A}_{D}.npz")


def make_sampled():
    for N, A, D in SAMPLED_GEOMS:
        t0 = time.time()
        f, yy = sampled_inputs(N, A, D)
        rng = np.random.default_rng(N * 31 + A * 7 + D)
        ai = rng.integers(0, A, N_SAMPLES).astype(np.int32)
        ii = rng.integers(0, D, N_SAMPLES).astype(np.int32)
        pix = rng.integers(0, N * N, N_SAMPLES).astype(np.int32)
        ys = oracle.radon_fwd_at(f.astype(np.float64), A, D, ai, ii)
        xs = oracle.radon_adj_at(yy.astype(np.float64), N, pix)
        np.savez_compressed(sampled_path(N, A, D), ai=ai, ii=ii, pix=pix, y=ys, x=xs)
        print(f"sampled {N} {A} {D}: {time.time() - t0:.1f} s", flush=True)


NOISY = dict(N=512, A=180, D=724, lam=1e-2, dims=2, iters=50, power_iters=12, i0=1e4)


def noisy_path():
    c = NOISY
    return os.path.join(HERE, f"noisy_{c['N']}_{c['A']}_{c['D']}.npz")


def make_noisy():
    c = NOISY
    N, A, D = c["N"], c["A"], c["D"]
    t0 = time.time()
    ells = synth.random_ellipses(N, synth.BASE_SEED + 512, scale=1.0 / N)
    p = synth.ellipse_line_integrals(ells, oracle.default_angles(A), D)[None]
    b, w = synth.poisson_measurement(p, c["i0"], synth.BASE_SEED + 513)
    b = b.astype(np.float32)
    w = w.astype(np.float32)
    b64, w64 = b.astype(np.float64), w.astype(np.float64)
    v0 = synth.random_start((1, N, N), synth.BASE_SEED + 514)
    lam_max = oracle.power_norm(N, A, D, w64, v0, c["power_iters"])
    step = 1.0 / (1.05 * lam_max + c["lam"] * oracle.prior_lipschitz(**oracle.PAPER_PRIOR))
    print(f"noisy: power iteration {time.time() - t0:.1f} s, lam_max {lam_max:.6g}, step {step:.6g}",
          flush=True)
    # the 10-iteration iterate is its own run from x_0 = 0 (the same schedule's
    # first ten steps)
    x10, log10 =oracle.mbir_solve(b64, w64, N, 10, step, lam=c["lam"], prior=oracle.PAPER_PRIOR,
                                   dims=c["dims"], return_log=True)
    print(f"noisy: 10 iterations {time.time() - t0:.1f} s", flush=True)
    x, log = oracle.mbir_solve(b64, w64, N, c["iters"], step, lam=c["lam"], prior=oracle.PAPER_PRIOR,
                               dims=c["dims"], return_log=True)
    np.savez_compressed(noisy_path(), b=b, w=w, step=step, lam_max=lam_max,
                        x10=x10.astype(np.float32), restarts10=sum(e["restart"] for e in log10),
                        x=x.astype(np.float32), restarts=sum(e["restart"] for e in log),
                        data=np.array([e["data"] for e in log]), prior=np.array([e["prior"] for e in log]))
    print(f"noisy: done {time.time() - t0:.1f} s, restarts {sum(e['restart'] for e in log)}", flush=True)


AUTOGRAD = dict(N=1024, A=360, D=1448, samples=512)


def autograd_inputs():
    c = AUTOGRAD
    N, A, D = c["N"], c["A"], c["D"]
    x = synth.uniform_field((N, N), synth.BASE_SEED + 1024)
    b = synth.uniform_field((A, D), synth.BASE_SEED + 1025, 0.0, 400.0)
    w = synth.uniform_field((A, D), synth.BASE_SEED + 1026, 0.2, 1.0)
    return x, b, w


def autograd_path():
    c = AUTOGRAD
    return os.path.join(HERE, f"autograd_{c['N']}_{c['A']}_{c['D']}.npz")


def make_autograd():
    c = AUTOGRAD
    N, A, D = c["N"], c["A"], c["D"]
    t0 = time.time()
    x, b, w = autograd_inputs()
    r = oracle.radon_fwd(x.astype(np.float64), A, D) - b.astype(np.float64)
    wr = w.astype(np.float64) * r
    loss = 0.5 * float(np.sum(wr * r))
    rng = np.random.default_rng(N + A + D)
    pix = rng.integers(0, N * N, c["samples"]).astype(np.int32)
    g = oracle.radon_adj_at(wr, N, pix)
    np.savez_compressed(autograd_path(), pix=pix, g=g, loss=loss)
    print(f"autograd: done {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    oracle.build()
    if what in ("sampled", "all"):
        make_sampled()
    if what in ("autograd", "all"):
        make_autograd()
    if what in ("noisy", "all"):
        make_noisy()
