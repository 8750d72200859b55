"""Seeded synthetic inputs shaped like synchrotron micro-CT data.

This module only draws inputs: random-ellipse phantoms, their analytic line
integrals (the continuous Radon transform of Sec. 2.1 Eq. radon_transform for
an ellipse, which no discrete operator here computes), Beer-Lambert/Poisson
measurements (Sec. 5: b = -log(I/I0)) and random start vectors.  It holds none
of the NUFFT or MBIR arithmetic, so the CUDA path and the FP64 oracle can both
take their inputs from it.

Phantom model (stand-in for the paper's foam phantom and Tomobank data, which
are not available here):
  * 10 ellipses per slice; centre uniform in the disk of radius 0.7 (units of
    N/2), semi-axes uniform in [0.05, 0.35] (units of N/2), orientation uniform
    in [0, pi), density uniform in [0, 1]; densities of overlapping ellipses add.
  * seed = 20230425 + slice index unless given.
  * pixel (ix, iy) has centre (ix - N/2, iy - N/2) and takes the summed density
    of the ellipses that contain that centre.
  * ``scale`` multiplies densities (1/N for the Poisson workloads, so that line
    integrals are O(1) and counts do not underflow).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20230425


@dataclass(frozen=True)
class Ellipse:
    cx: float      # centre, pixel units relative to the image centre
    cy: float
    a: float       # semi-axes, pixels
    b: float
    phi: float     # orientation of the a-axis, radians
    rho: float     # density (attenuation per pixel length)


def random_ellipses(n: int, seed: int, n_ellipses: int = 10, scale: float = 1.0):
    rng = np.random.default_rng(seed)
    h = n / 2.0
    out = []
    for _ in range(n_ellipses):
        r = 0.7 * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        a, b = rng.uniform(0.05, 0.35, size=2)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        out.append(Ellipse(r * math.cos(ang) * h, r * math.sin(ang) * h,
                           a * h, b * h, phi, rho * scale))
    return out


def rasterize(n: int, ellipses) -> np.ndarray:
    """Image [n, n] (row = iy, column = ix) with summed ellipse densities."""
    c = np.arange(n, dtype=np.float64) - n // 2
    X, Y = np.meshgrid(c, c)  # X[iy, ix] = ix - n/2
    img = np.zeros((n, n), np.float64)
    for e in ellipses:
        dx, dy = X - e.cx, Y - e.cy
        cp, sp = math.cos(e.phi), math.sin(e.phi)
        u = dx * cp + dy * sp
        v = -dx * sp + dy * cp
        img[(u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0] += e.rho
    return img


def ellipse_line_integrals(ellipses, theta, n_det: int) -> np.ndarray:
    """Analytic sinogram [A, D]: integral of the phantom along the line
    <x, (cos th, sin th)> = t_i, t_i = i - D/2 (Sec. 2.1 Eq. line_eqn)."""
    theta = np.asarray(theta, np.float64)
    t = np.arange(n_det, dtype=np.float64) - n_det // 2
    out = np.zeros((theta.shape[0], n_det), np.float64)
    for e in ellipses:
        r2 = (e.a * np.cos(theta - e.phi)) ** 2 + (e.b * np.sin(theta - e.phi)) ** 2
        tc = e.cx * np.cos(theta) + e.cy * np.sin(theta)
        d = t[None, :] - tc[:, None]
        rem = r2[:, None] - d * d
        out += np.where(rem > 0, 2.0 * e.rho * e.a * e.b * np.sqrt(np.maximum(rem, 0.0)) / r2[:, None], 0.0)
    return out


def gaussian_blob(n: int, cx: float, cy: float, s: float, amp: float = 1.0) -> np.ndarray:
    c = np.arange(n, dtype=np.float64) - n // 2
    X, Y = np.meshgrid(c, c)
    return amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s * s))


def gaussian_line_integrals(cx, cy, s, theta, n_det, amp=1.0) -> np.ndarray:
    """Analytic projection of amp*exp(-|x-c|^2/(2 s^2)): sqrt(2 pi) s amp
    exp(-(t - <c, n>)^2 / (2 s^2))."""
    theta = np.asarray(theta, np.float64)
    t = np.arange(n_det, dtype=np.float64) - n_det // 2
    tc = cx * np.cos(theta) + cy * np.sin(theta)
    return amp * math.sqrt(2.0 * math.pi) * s * np.exp(-(t[None, :] - tc[:, None]) ** 2 / (2.0 * s * s))


def poisson_measurement(p_true: np.ndarray, i0: float, seed: int):
    """Beer-Lambert counts I ~ Poisson(I0 exp(-p)), clamped to I >= 1.

    Returns (b, w) with b = -log(I/I0) (Sec. 5) and weights w = I/I0
    (proportional to counts).
    """
    rng = np.random.default_rng(seed)
    counts = rng.poisson(i0 * np.exp(-p_true)).astype(np.float64)
    counts = np.maximum(counts, 1.0)
    return -np.log(counts / i0), counts / i0


def random_start(shape, seed: int) -> np.ndarray:
    """Seeded normal start vector (power iteration / finite differences)."""
    return np.random.default_rng(seed).standard_normal(shape)


def phantom_slices(n: int, n_slices: int, scale: float = 1.0, seed0: int = BASE_SEED):
    """[B, n, n] stack of independent random-ellipse slices plus their ellipses."""
    ells = [random_ellipses(n, seed0 + k, scale=scale) for k in range(n_slices)]
    return np.stack([rasterize(n, e) for e in ells]), ells


def ellipsoid_volume_slices(n: int, nz: int, z_index, n_ellipsoids: int = 10,
                            scale: float = 1.0, seed: int = BASE_SEED):
    """Slices of a 3D phantom of ellipsoids rotated about z only.

    Each ellipsoid has centre (cx, cy, cz), semi-axes (a, b, c) and rotation
    phi about z, all seeded; slice z cuts it in an exact ellipse with
    semi-axes scaled by sqrt(1 - ((z - cz)/c)^2).  Returns the list of
    ellipse lists, one per requested slice index (the volume itself can be
    rasterized slice by slice on demand).
    """
    rng = np.random.default_rng(seed)
    h = n / 2.0
    hz = nz / 2.0
    bodies = []
    for _ in range(n_ellipsoids):
        r = 0.7 * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        a, b = rng.uniform(0.05, 0.35, size=2)
        cz = rng.uniform(-0.6, 0.6)
        c = rng.uniform(0.1, 0.4)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        bodies.append((r * math.cos(ang) * h, r * math.sin(ang) * h, cz * hz,
                       a * h, b * h, c * hz, phi, rho * scale))
    out = []
    for z in z_index:
        zc = z - nz // 2
        ells = []
        for cx, cy, cz, a, b, c, phi, rho in bodies:
            q = 1.0 - ((zc - cz) / c) ** 2
            if q > 0:
                k = math.sqrt(q)
                ells.append(Ellipse(cx, cy, a * k, b * k, phi, rho))
        out.append(ells)
    return out


# ------------------------------------------------------------- workloads ----
@dataclass(frozen=True)
class Workload:
    name: str
    n: int          # image side N
    n_angles: int   # A
    n_det: int      # D
    slices: int     # B
    n_iter: int
    noise_i0: float | None   # Poisson I0, None = noise-free analytic data
    prior_dims: int          # 2: 8 in-plane neighbours, 3: 26 neighbours


# Sizes of the five synthetic workloads (slices, angles, detector bins).
WORKLOADS = {
    "single_128": Workload("single_128", 128, 90, 184, 1, 20, None, 2),
    "noisy_512x16": Workload("noisy_512x16", 512, 180, 724, 16, 50, 1e4, 2),
    "diff_1024x64": Workload("diff_1024x64", 1024, 360, 1448, 64, 0, None, 3),
    "volume_2048x1024": Workload("volume_2048x1024", 2048, 128, 2896, 1024, 100, 1e4, 3),
    # shapes of the paper's two real-data experiments (Sec. 5), as synthetic
    # stand-ins: 400 projections x 2048 bins and 202 projections x 2448 bins,
    # 128 slices each, reconstructed on a 2048^2 grid
    "tb25_shape": Workload("tb25_shape", 2048, 400, 2048, 128, 100, 1e4, 3),
    "tb86_shape": Workload("tb86_shape", 2048, 202, 2448, 128, 100, 1e4, 3),
}


def det_for(n: int) -> int:
    """Detector width for a side n: 2*round(n/sqrt 2) (covers the image disk)."""
    return 2 * int(round(n / math.sqrt(2.0)))


# ------------------------------------------------- large volumes (torch) ----
def ellipsoid_bodies(n: int, nz: int, n_ellipsoids: int = 10, scale: float = 1.0,
                     seed: int = BASE_SEED):
    """Seeded ellipsoids rotated about z only (same draws as
    ellipsoid_volume_slices): rows (cx, cy, cz, a, b, c, phi, rho)."""
    rng = np.random.default_rng(seed)
    h, hz = n / 2.0, nz / 2.0
    rows = []
    for _ in range(n_ellipsoids):
        r = 0.7 * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        a, b = rng.uniform(0.05, 0.35, size=2)
        cz = rng.uniform(-0.6, 0.6)
        c = rng.uniform(0.1, 0.4)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        rows.append((r * math.cos(ang) * h, r * math.sin(ang) * h, cz * hz,
                     a * h, b * h, c * hz, phi, rho * scale))
    return np.array(rows, dtype=np.float64)


def ellipsoid_sinogram_torch(n, nz, theta, n_det, device, scale=1.0, seed=BASE_SEED,
                             z_chunk=64):
    """Analytic line integrals [nz, A, D] (float32, on `device`) of the
    ellipsoid phantom: slice z of an ellipsoid is an ellipse with semi-axes
    scaled by k = sqrt(1 - ((z - cz)/c)^2), whose projection is
    2 rho a b sqrt(k^2 r^2 - d^2) / r^2, r^2 = a^2 cos^2(th - phi) + b^2 sin^2(th - phi)."""
    import torch
    bodies = ellipsoid_bodies(n, nz, scale=scale, seed=seed)
    th = torch.as_tensor(np.asarray(theta, np.float64), device=device)
    t = torch.arange(n_det, device=device, dtype=torch.float64) - n_det // 2
    out = torch.empty((nz, th.shape[0], n_det), device=device, dtype=torch.float32)
    zc = torch.arange(nz, device=device, dtype=torch.float64) - nz // 2
    for z0 in range(0, nz, z_chunk):
        z1 = min(nz, z0 + z_chunk)
        acc = torch.zeros((z1 - z0, th.shape[0], n_det), device=device, dtype=torch.float64)
        for cx, cy, cz, a, b, c, phi, rho in bodies:
            k2 = (1.0 - ((zc[z0:z1] - cz) / c) ** 2).clamp(min=0.0)
            r2 = (a * torch.cos(th - phi)) ** 2 + (b * torch.sin(th - phi)) ** 2
            tc = cx * torch.cos(th) + cy * torch.sin(th)
            d = t[None, :] - tc[:, None]
            rem = k2[:, None, None] * r2[None, :, None] - (d * d)[None]
            acc += 2.0 * rho * a * b * torch.sqrt(rem.clamp(min=0.0)) / r2[None, :, None]
        out[z0:z1] = acc.float()
    return out


def poisson_measurement_torch(p_true, i0: float, seed: int):
    """Torch version of poisson_measurement (same model, on p_true's device)."""
    import torch
    g = torch.Generator(device=p_true.device)
    g.manual_seed(seed)
    counts = torch.poisson((i0 * torch.exp(-p_true.double())), generator=g).clamp_(min=1.0)
    return (-torch.log(counts / i0)).float(), (counts / i0).float()


# ------------------------------------------------- platform-exact fields ----
def uniform_field(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Seeded float32 array, uniform in [lo, hi).  The draw uses only integer
    generator output and exact scaling (no libm), so it is bit-identical on
    every platform: stored expected values computed on one machine stay valid
    on another."""
    u = np.random.default_rng(seed).random(shape)
    return (lo + (hi - lo) * u).astype(np.float32)
