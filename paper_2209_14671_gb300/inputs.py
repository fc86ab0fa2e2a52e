"""Seeded synthetic inputs for the Elfpie workloads.

This module is the only one read by both the CUDA path and the FP64 oracle.  It
holds no arithmetic of the method: it draws LED geometries (Sec. 4.1's physical
set-up), smooth random complex objects standing in for the paper's Fig. 3
images, and the degradations of Eq. 2 / Eq. 20 applied to an already simulated
clean intensity.  The forward model itself (crop, pupil, inverse FFT, |.|^2) is
applied by each side with its own code.

Random streams are NumPy PCG64 seeded ``default_rng([workload_id, stream])``:
0 amplitude, 1 phase, 2 Gaussian noise, 3 salt & pepper, 4 Poisson, 5 background,
6 LED jitter, 7 finite-difference directions, 8 serving arrivals, 9 state
perturbation for parity tests.
"""
from __future__ import annotations

import math

import numpy as np

STREAM_AMP, STREAM_PHASE, STREAM_NOISE, STREAM_SNP, STREAM_POISSON = 0, 1, 2, 3, 4
STREAM_BG, STREAM_JITTER, STREAM_FD, STREAM_ARRIVALS, STREAM_STATE = 5, 6, 7, 8, 9

# Workload recipes.  Sizes: n low-res side, u upsampling (N = u n), LED grid side.
WORKLOADS = {
    # 7x7 LEDs, 64x64 images, 256x256 object, sigma 1e-3 Gaussian noise, 20 iterations
    0: dict(name="plain_n64_N256_K49", n=64, u=4, grid=7, pitch_mm=4.0, height_mm=90.0,
            na=0.1, wavelength_um=0.63, pixel_um=1.625, iters=20,
            noise=dict(gauss_sigma=1e-3)),
    # Sec. 4.1 geometry at 256x256 images, 1024x1024 object, 15x15 LEDs, mixed corruptions
    1: dict(name="degraded_n256_N1024_K225", n=256, u=4, grid=15, pitch_mm=6.0, height_mm=90.0,
            na=0.1, wavelength_um=0.536, pixel_um=3.65 / 4.0, iters=100,
            noise=dict(gauss_sigma_max=0.1, photons=1e3, snp_density=0.05,
                       background_max=0.1, vignette_ring=7, jitter_mm=2.0)),
    # differentiation check at workload-0 sizes
    2: dict(name="diffcheck_n64_N256_K49", n=64, u=4, grid=7, pitch_mm=4.0, height_mm=90.0,
            na=0.1, wavelength_um=0.63, pixel_um=1.625, iters=0,
            noise=dict(gauss_sigma=1e-3)),
    # Sec. 4.1 geometry at 128x128 images, 512x512 object, 15x15 LEDs, 200 iterations
    3: dict(name="precision_n128_N512_K225", n=128, u=4, grid=15, pitch_mm=6.0, height_mm=90.0,
            na=0.1, wavelength_um=0.536, pixel_um=3.65 / 4.0, iters=200,
            noise=dict(gauss_sigma=1e-3)),
}


def rng(workload_id: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(workload_id), int(stream)])


def led_positions_mm(grid: int, pitch_mm: float) -> np.ndarray:
    """[K, 2] (x, y) LED positions of a square grid centred on the optical axis.
    Order: row-major, y outer, x inner, both ascending."""
    idx = (np.arange(grid) - (grid - 1) / 2.0) * pitch_mm
    yy, xx = np.meshgrid(idx, idx, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def kxy_from_positions(pos_mm: np.ndarray, height_mm: float, wavelength_um: float) -> np.ndarray:
    """Illumination spatial frequency (kx, ky) = (sin theta_x, sin theta_y)/lambda, cycles/um."""
    pos = np.asarray(pos_mm, dtype=np.float64)
    r = np.sqrt(pos[:, 0] ** 2 + pos[:, 1] ** 2 + height_mm ** 2)
    return np.stack([pos[:, 0] / r, pos[:, 1] / r], axis=1) / wavelength_um


def problem(workload_id: int, grid: int | None = None, n: int | None = None) -> dict:
    """Geometry of a workload: nominal k (for reconstruction) and true k (for simulation).

    ``grid`` and ``n`` override the LED grid side and image size (serving mixes)."""
    w = dict(WORKLOADS[workload_id])
    if grid is not None:
        w["grid"] = int(grid)
    if n is not None:
        w["n"] = int(n)  # same optics and pixel size; the spectral pixel scales as 1/n
    pos = led_positions_mm(w["grid"], w["pitch_mm"])
    k_nom = kxy_from_positions(pos, w["height_mm"], w["wavelength_um"])
    jit = w["noise"].get("jitter_mm", 0.0)
    if jit:
        d = rng(workload_id, STREAM_JITTER).uniform(-jit, jit, size=pos.shape)
        k_true = kxy_from_positions(pos + d, w["height_mm"], w["wavelength_um"])
    else:
        k_true = k_nom.copy()
    w["N"] = w["n"] * w["u"]
    w["K"] = int(pos.shape[0])
    w["k_xy"] = k_nom
    w["k_xy_true"] = k_true
    return w


def object_sigma_px(w: dict) -> float:
    """Smoothness of the synthetic object, in spectral pixels: 0.6 x (largest LED
    frequency along one axis + pupil radius), both measured in units of 1/(n dx)."""
    dk = 1.0 / (w["n"] * w["pixel_um"])
    kmax = float(np.max(np.abs(w["k_xy"])))
    return 0.6 * (kmax + w["na"] / w["wavelength_um"]) / dk


def smooth_field(N: int, sigma_px: float, g: np.random.Generator) -> np.ndarray:
    """White Gaussian noise low-passed by exp(-|f|^2 / (2 sigma^2)) and scaled to [0, 1]."""
    white = g.standard_normal((N, N))
    f = np.fft.fftfreq(N) * N
    filt = np.exp(-(f[None, :] ** 2 + f[:, None] ** 2) / (2.0 * sigma_px ** 2))
    field = np.real(np.fft.ifft2(np.fft.fft2(white) * filt))
    lo, hi = field.min(), field.max()
    return (field - lo) / (hi - lo)


def object_field(workload_id: int, w: dict | None = None) -> np.ndarray:
    """Complex object: amplitude in [0.2, 1], phase in [-pi/2, pi/2] (complex128 [N, N])."""
    w = w or problem(workload_id)
    s = object_sigma_px(w)
    amp = 0.2 + 0.8 * smooth_field(w["N"], s, rng(workload_id, STREAM_AMP))
    ph = (smooth_field(w["N"], s, rng(workload_id, STREAM_PHASE)) - 0.5) * math.pi
    return amp * np.exp(1j * ph)


def corrupt(I_clean: np.ndarray, workload_id: int, w: dict | None = None) -> np.ndarray:
    """Degrade clean intensities [K, n, n] with the workload's recipe (Eqs. 2, 20).

    Order: vignetting (outer LED ring), Poisson photon counting, per-LED background,
    Gaussian noise, salt & pepper (half to 1, half to 0).  Returns float32."""
    w = w or problem(workload_id)
    nz = w["noise"]
    I = np.array(I_clean, dtype=np.float64, copy=True)
    K, n, _ = I.shape
    if "vignette_ring" in nz:
        half = (w["grid"] - 1) // 2
        ring = nz["vignette_ring"]
        yy, xx = np.meshgrid(np.arange(n) - n / 2, np.arange(n) - n / 2, indexing="ij")
        rho2 = (xx ** 2 + yy ** 2) / (n / 2.0) ** 2
        lam = np.clip(1.0 - 0.5 * rho2, 0.0, 1.0)
        for k in range(K):
            iy, ix = divmod(k, w["grid"])
            if max(abs(iy - half), abs(ix - half)) == ring:
                I[k] *= lam
    if "photons" in nz:
        ph = nz["photons"]
        I = rng(workload_id, STREAM_POISSON).poisson(np.maximum(I, 0.0) * ph) / ph
    if "background_max" in nz:
        bg = rng(workload_id, STREAM_BG).uniform(0.0, nz["background_max"], size=K)
        I += bg[:, None, None]
    g = rng(workload_id, STREAM_NOISE)
    if "gauss_sigma" in nz:
        I += nz["gauss_sigma"] * g.standard_normal(I.shape)
    if "gauss_sigma_max" in nz:
        sig = g.uniform(0.0, nz["gauss_sigma_max"], size=K)
        I += sig[:, None, None] * g.standard_normal(I.shape)
    if "snp_density" in nz:
        h = rng(workload_id, STREAM_SNP)
        m = h.random(I.shape) < nz["snp_density"]
        salt = h.random(I.shape) < 0.5
        I = np.where(m, np.where(salt, 1.0, 0.0), I)
    return I.astype(np.float32)


def complex_directions(shape, count: int, workload_id: int) -> np.ndarray:
    """Seeded complex unit-norm directions for finite-difference checks, [count, *shape]."""
    g = rng(workload_id, STREAM_FD)
    d = g.standard_normal((count,) + tuple(shape)) + 1j * g.standard_normal((count,) + tuple(shape))
    norms = np.sqrt(np.sum(np.abs(d) ** 2, axis=tuple(range(1, d.ndim)), keepdims=True))
    return d / norms
