"""Shared problem builders for the parity tests.

Inputs come from the seeded generator (paper_2209_14671_gb300.inputs); the clean
intensities are simulated by the FP64 oracle's forward model, so both the CUDA
path and the oracle see exactly the same float32 measurements.
"""
from __future__ import annotations

import functools

import numpy as np

import oracle as O
from paper_2209_14671_gb300 import inputs as IN


def _tiny(n, u, grid, step, na_px, seed, sigma=1e-3):
    dk = 1.0 / n
    c = (np.arange(grid) - (grid - 1) // 2) * step
    cy, cx = np.meshgrid(c, c, indexing="ij")
    k_xy = np.stack([cx.ravel() * dk, cy.ravel() * dk], axis=1)
    na, wl, dx = na_px * dk, 1.0, 1.0
    geo = O.make_geometry(n, u, k_xy, na, wl, dx)
    N = n * u
    g = np.random.default_rng(seed)
    f = np.fft.fftfreq(N) * N
    filt = np.exp(-(f[None, :] ** 2 + f[:, None] ** 2) / (2 * (N / 8.0) ** 2))

    def field():
        x = np.real(np.fft.ifft2(np.fft.fft2(g.standard_normal((N, N))) * filt))
        return (x - x.min()) / (x.max() - x.min())
    obj = (0.3 + 0.7 * field()) * np.exp(1j * (field() - 0.5) * 2.0)
    I = O.forward_intensity(O.spectrum_from_object(obj), geo.support.astype(complex), geo)
    I = (I + sigma * g.standard_normal(I.shape)).astype(np.float32)
    return dict(name=f"tiny_n{n}_u{u}_K{grid * grid}", n=n, u=u, k_xy=k_xy, na=na, wl=wl, dx=dx,
                geo=geo, obj=obj, I=I)


def _workload(w):
    p = IN.problem(w)
    geo_true = O.make_geometry(p["n"], p["u"], p["k_xy_true"], p["na"], p["wavelength_um"], p["pixel_um"])
    geo = O.make_geometry(p["n"], p["u"], p["k_xy"], p["na"], p["wavelength_um"], p["pixel_um"])
    obj = IN.object_field(w, p)
    I_clean = O.forward_intensity(O.spectrum_from_object(obj), geo_true.support.astype(complex), geo_true)
    I = IN.corrupt(I_clean, w, p)
    return dict(name=p["name"], n=p["n"], u=p["u"], k_xy=p["k_xy"], na=p["na"], wl=p["wavelength_um"],
                dx=p["pixel_um"], geo=geo, obj=obj, I=I, iters=p["iters"], k_xy_true=p["k_xy_true"])


@functools.lru_cache(maxsize=None)
def case(name: str) -> dict:
    if name == "tiny16":
        return _tiny(16, 2, 3, 4, 5.0, 1)
    if name == "small32":
        return _tiny(32, 4, 5, 5, 7.5, 2)
    if name == "single_led":
        return _tiny(32, 2, 1, 0, 6.0, 3)
    if name == "nou32":  # no upsampling (u = 1): the one LED's crop is the whole spectrum
        return _tiny(32, 1, 1, 0, 6.0, 5)
    if name == "wide256":  # n = 256 with a pupil band of 231 rows: the widest tile-kernel shared memory layout
        return _tiny(256, 2, 3, 40, 115.0, 4)
    if name.startswith("w"):
        return _workload(int(name[1:]))
    raise KeyError(name)


def oracle_state_to_f32(st: O.State) -> O.State:
    """Round an oracle state to the float32 the GPU holds, back in float64."""
    s = st.copy()
    for k in ("psi", "mu_psi", "pupil", "mu_p"):
        setattr(s, k, getattr(s, k).astype(np.complex64).astype(np.complex128))
    for k in ("v_psi", "delta_psi", "v_p", "delta_p"):
        setattr(s, k, getattr(s, k).astype(np.float32).astype(np.float64))
    return s


def load_state(elf, st: O.State):
    elf.set_state(st.psi, st.mu_psi, st.v_psi, st.delta_psi, st.pupil, st.mu_p, st.v_p, st.delta_p,
                  st.t, st.alpha, st.beta)


def rel(a, b) -> float:
    nb = np.linalg.norm(np.asarray(b).ravel())
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / (nb if nb > 0 else 1.0))
