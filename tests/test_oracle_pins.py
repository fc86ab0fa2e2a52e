"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the DFT
definition summed by brute force, Parseval, exact adjoint identities, central
finite differences, the affine null space of the Hessian, closed forms for
Eq. 16 and for Eq. 19, a zero gradient at the true state, noiseless convergence,
and the constants the paper prints (tests/golden/paper_constants.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# --------------------------------------------------------------------------- helpers
def tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0, mux=1, extra_leds=0):
    """Geometry with exact integer LED offsets (k = c * dk) and a pupil of radius na_px;
    `extra_leds` repeats the first LEDs at the end so that K is a multiple of `mux`."""
    dk = 1.0 / n  # pixel 1 um
    c = (np.arange(grid) - (grid - 1) // 2) * step
    cy, cx = np.meshgrid(c, c, indexing="ij")
    k_xy = np.stack([cx.ravel() * dk, cy.ravel() * dk], axis=1)
    if extra_leds:
        k_xy = np.concatenate([k_xy, k_xy[:extra_leds] + 0.5 * dk], axis=0)
    geo = O.make_geometry(n, u, k_xy, na=na_px * dk, wavelength_um=1.0, pixel_um=1.0, mux=mux)
    return geo, k_xy


def smooth_object(N, seed, amp=(0.3, 1.0), ph=(-1.0, 1.0), sigma=4.0):
    g = np.random.default_rng(seed)
    f = np.fft.fftfreq(N) * N
    filt = np.exp(-(f[None, :] ** 2 + f[:, None] ** 2) / (2 * sigma ** 2))

    def field():
        x = np.real(np.fft.ifft2(np.fft.fft2(g.standard_normal((N, N))) * filt))
        return (x - x.min()) / (x.max() - x.min())
    a = amp[0] + (amp[1] - amp[0]) * field()
    p = ph[0] + (ph[1] - ph[0]) * field()
    return a * np.exp(1j * p)


def centred(k, n):
    """centred spectral index -> frequency (index - n/2)."""
    return k - n // 2


# --------------------------------------------------------------------------- constants
def test_constants_match_paper():
    gold = json.load(open(GOLDEN))
    assert np.array_equal(O.LAPLACE_KERNEL, np.array(gold["laplace_kernel"]["value"], float))
    opt = O.Options()
    assert opt.gamma1 == gold["gamma1_default"]["value"]
    assert opt.gamma2 == gold["gamma2_default"]["value"]
    assert opt.s0_psi ** 2 == gold["delta0"]["value"]
    k = O.gauss3()
    assert k.shape == (gold["pupil_filter"]["size"],) * 2
    # sigma = 1 px: the ratio of an edge weight to the centre weight is exp(-1/2)
    assert math.isclose(k[1, 0] / k[1, 1], math.exp(-0.5 / gold["pupil_filter"]["sigma_px"] ** 2))
    assert math.isclose(k.sum(), 1.0)


def test_round_half_away_and_support():
    assert list(O.round_half_away([2.5, -2.5, 0.49, -0.51, 1.5])) == [3, -3, 0, -1, 2]
    geo, _ = tiny_problem(n=16, na_px=5.0)
    # explicit count of integer points with jx^2 + jy^2 <= 25
    cnt = sum(1 for a in range(-8, 8) for b in range(-8, 8) if a * a + b * b <= 25)
    assert geo.support.sum() == cnt == 81
    assert geo.support[8, 8] and geo.support[8, 13] and not geo.support[8, 14]


def test_geometry_offsets_round_half_away():
    dk = 1.0 / 16
    geo = O.make_geometry(16, 2, [[2.5 * dk, -2.5 * dk], [-0.5 * dk, 1.5 * dk]], na=0.2,
                          wavelength_um=1.0, pixel_um=1.0)
    assert geo.offsets.tolist() == [[-3, 3], [2, -1]]
    assert geo.origins.tolist() == [[16 - 8 - 3, 16 - 8 + 3], [16 - 8 + 2, 16 - 8 - 1]]


def test_geometry_rejects_out_of_range_window():
    with pytest.raises(ValueError):
        O.make_geometry(16, 2, [[20 / 16.0, 0.0]], na=0.2, wavelength_um=1.0, pixel_um=1.0)


# --------------------------------------------------------------------------- transforms (A1)
@pytest.mark.parametrize("N", [4, 6, 8])
def test_object_from_spectrum_is_the_centred_idft(N):
    g = np.random.default_rng(N)
    psi = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    # definition: O[y,x] = (1/A) sum_k Psi[k] exp(2 pi i (k - N/2).x / N)
    want = np.zeros((N, N), complex)
    for y in range(N):
        for x in range(N):
            for ky in range(N):
                for kx in range(N):
                    want[y, x] += psi[ky, kx] * np.exp(
                        2j * np.pi * (centred(ky, N) * y + centred(kx, N) * x) / N)
    want /= N * N
    assert np.allclose(O.object_from_spectrum(psi), want, atol=1e-13)
    assert np.allclose(O.spectrum_from_object(O.object_from_spectrum(psi)), psi, atol=1e-12)


def test_forward_field_brute_force():
    geo, _ = tiny_problem(n=8, u=2, grid=1, na_px=3.0)
    g = np.random.default_rng(1)
    psi = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
    pupil = g.standard_normal((8, 8)) + 1j * g.standard_normal((8, 8))
    t = (pupil * geo.support) * psi[4:12, 4:12]
    # o[y,x] = u^-2 (1/B) sum_j t[j] exp(2 pi i (j - n/2).x / n)
    want = np.zeros((8, 8), complex)
    for y in range(8):
        for x in range(8):
            for jy in range(8):
                for jx in range(8):
                    want[y, x] += t[jy, jx] * np.exp(2j * np.pi * ((jy - 4) * y + (jx - 4) * x) / 8)
    want /= 64 * 4
    assert np.allclose(O.forward_field(psi, pupil, geo, 0), want, atol=1e-13)


def test_plane_wave_and_uniform_object():
    N = 16
    psi = np.zeros((N, N), complex)
    psi[N // 2 + 3, N // 2 - 2] = 1.0
    obj = O.object_from_spectrum(psi)
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    assert np.allclose(obj, np.exp(2j * np.pi * (3 * yy - 2 * xx) / N) / (N * N), atol=1e-15)
    # uniform object through the on-axis LED with P(0)=1 images to itself (u^-2 scaling)
    geo, _ = tiny_problem(n=8, u=2, grid=1, na_px=2.0)
    obj = np.full((16, 16), 0.7 - 0.2j)
    o = O.forward_field(O.spectrum_from_object(obj), np.ones((8, 8)), geo, 0)
    assert np.allclose(o, 0.7 - 0.2j, atol=1e-13)


def test_parseval():
    g = np.random.default_rng(3)
    obj = g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))
    psi = O.spectrum_from_object(obj)
    assert math.isclose(np.sum(np.abs(psi) ** 2), 32 * 32 * np.sum(np.abs(obj) ** 2), rel_tol=1e-12)


# --------------------------------------------------------------------------- adjoints
def _inner(a, b):
    return np.vdot(a, b)


def test_adjoint_identities():
    g = np.random.default_rng(5)
    r = g.standard_normal((12, 9))
    px, py = g.standard_normal((12, 9)), g.standard_normal((12, 9))
    gx, gy = O.grad_op(r)
    assert math.isclose(np.sum(gx * px) + np.sum(gy * py), np.sum(r * O.grad_adj(px, py)), rel_tol=1e-12)
    f = g.standard_normal((11, 13))
    w = [g.standard_normal((11, 13)) for _ in range(3)]
    for c in w:  # H^T is applied to fields living on the interior
        c[0, :] = c[-1, :] = 0
        c[:, 0] = c[:, -1] = 0
    h = O.hessian_op(f)
    lhs = sum(np.sum(a * b) for a, b in zip(h, w))
    assert math.isclose(lhs, np.sum(f * O.hessian_adj(*w)), rel_tol=1e-12)
    p = g.standard_normal((10, 10)) + 1j * g.standard_normal((10, 10))
    q = g.standard_normal((10, 10)) + 1j * g.standard_normal((10, 10))
    assert abs(_inner(O.filter3(p), q) - _inner(p, O.filter3(q))) < 1e-12
    geo, _ = tiny_problem(n=8, u=2, grid=3, step=2, na_px=3.0)
    big = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
    small = g.standard_normal((8, 8)) + 1j * g.standard_normal((8, 8))
    for k in range(geo.K):
        assert abs(_inner(O.crop(big, geo, k), small) - _inner(big, O.crop_adjoint(small, geo, k))) < 1e-12


def test_fidelity_gradient_is_adjoint_of_forward_operator():
    """With tau huge, phi = |d|^2/(2 tau) + tau/2 is quadratic, so the gradient of the
    intensity fidelity must equal the explicit chain of adjoints built term by term."""
    geo, _ = tiny_problem(n=8, u=2, grid=3, step=2, na_px=3.0)
    opt = O.Options(tau_fid=1e6)
    obj = smooth_object(16, 2)
    psi = O.spectrum_from_object(obj)
    pupil = np.exp(0.3j) * np.ones((8, 8))
    I = np.random.default_rng(4).uniform(0, 1, (geo.K, 8, 8))
    _, g_psi, g_p, _ = O.fidelity_cost_grad(psi, pupil, I, geo, opt)
    # explicit T_n and T_n^H as dense matrices on the 8x8 tile (independent of fft helpers)
    n = 8
    j = np.arange(n) - n // 2
    E = np.exp(2j * np.pi * np.outer(np.arange(n), j) / n) / n    # x <- centred j, 1D
    want = np.zeros_like(psi)
    for k in range(geo.K):
        t = (pupil * geo.support) * O.crop(psi, geo, k)
        o = E @ t @ E.T / 4.0
        r = np.abs(o) ** 2 - I[k]
        dx, dy = O.grad_op(r)
        w = O.grad_adj(dx / 1e6, dy / 1e6)
        W = o * w
        G = E.conj().T @ W @ E.conj() / 4.0
        want += O.crop_adjoint(np.conj(pupil * geo.support) * G, geo, k)
    assert np.allclose(g_psi, want, atol=1e-12 * np.abs(want).max())


# --------------------------------------------------------------------------- finite differences
def _total(psi, pupil, I, geo, opt, alpha, beta):
    L_fid, _, _, _ = O.fidelity_cost_grad(psi, pupil, I, geo, opt)
    L_A, L_P, _ = O.hessian_cost_grad(psi, alpha, beta, opt)
    return L_fid + alpha * L_A + beta * L_P


FD_STEPS = (1e-3, 1e-4, 1e-5, 1e-6, 1e-7)
FD_DIRECTIONS = 32
FD_TOL = 1e-6


def fd_worst_error(f, x, g, rng, mask=None, n_dir=FD_DIRECTIONS, steps=FD_STEPS):
    """Central differences of the real function f along n_dir seeded complex directions d
    (scaled to ||d|| = ||x||), (f(x + h d) - f(x - h d)) / (2h) against the Wirtinger form
    2 Re<g, d> of the derivative, with h scanned over `steps`.  Per direction the error is the
    smallest over h, measured against |2 Re<g, d>| or, for a direction that happens to be nearly
    orthogonal to g, against the typical size 2 ||g|| ||d|| / sqrt(2m) of that derivative for a
    random direction in m complex dimensions.  Returns the worst direction's error."""
    m = int(np.count_nonzero(mask)) if mask is not None else x.size
    worst = 0.0
    for _ in range(n_dir):
        d = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        if mask is not None:
            d = d * mask
        d *= np.linalg.norm(x) / np.linalg.norm(d)
        an = 2.0 * np.real(np.vdot(g, d))
        scale = max(abs(an), 2.0 * np.linalg.norm(g) * np.linalg.norm(d) / math.sqrt(2.0 * m))
        err = min(abs((f(x + h * d) - f(x - h * d)) / (2 * h) - an) for h in steps) / scale
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("fidelity,iso,gexp", [(0, 1, 1.0), (1, 1, 1.0), (0, 0, 1.0), (2, 1, 0.375),
                                               (2, 0, 1.75), (3, 1, 1.0)])
def test_gradient_matches_central_differences(fidelity, iso, gexp):
    """Eqs. 9-14 and 18 (with the fidelity of Eq. 5, Eq. 4 or a Sec. 6.3 map) against central
    differences of Eq. 8 along 32 seeded complex directions each for Psi and P, h scanned over
    1e-3 .. 1e-7: agreement to 1e-6."""
    geo, k_xy = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)
    opt = O.Options(fidelity=fidelity, omega_iso=iso, tau_fid=1e-3, tau_h=1e-3, g_exponent=gexp)
    truth = smooth_object(geo.N, 11)
    I = O.forward_intensity(O.spectrum_from_object(truth), np.ones((16, 16)), geo)
    I = I + 0.01 * np.random.default_rng(12).standard_normal(I.shape)
    psi = O.spectrum_from_object(smooth_object(geo.N, 13))
    pupil = geo.support * np.exp(0.2j * np.random.default_rng(14).standard_normal((16, 16)))
    alpha, beta = 0.05, 0.03
    _, g_fid, g_p, _ = O.fidelity_cost_grad(psi, pupil, I, geo, opt)
    _, _, g_h = O.hessian_cost_grad(psi, alpha, beta, opt)
    rng = np.random.default_rng(15)
    e_psi = fd_worst_error(lambda x: _total(x, pupil, I, geo, opt, alpha, beta), psi, g_fid + g_h, rng)
    e_p = fd_worst_error(lambda x: _total(psi, x, I, geo, opt, alpha, beta), pupil, g_p, rng, mask=geo.support)
    print(f"worst of 32 directions: Psi {e_psi:.1e}, P {e_p:.1e}")
    assert e_psi <= FD_TOL and e_p <= FD_TOL


def test_zero_gradient_at_the_true_state():
    """Noiseless data generated by the same model: r = 0, omega = 0, so W = 0."""
    geo, _ = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)
    opt = O.Options()
    truth = O.spectrum_from_object(smooth_object(geo.N, 21))
    pupil = geo.support.astype(complex)
    I = O.forward_intensity(truth, pupil, geo)
    L, g_psi, g_p, _ = O.fidelity_cost_grad(truth, pupil, I, geo, opt)
    assert math.isclose(L, geo.K * 16 * 16 * opt.tau_fid / 2, rel_tol=1e-6)
    assert np.abs(g_psi).max() < 1e-9 * np.abs(truth).max()
    assert np.abs(g_p).max() < 1e-9


def _fid_problem(seed):
    geo, _ = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)
    truth = smooth_object(geo.N, seed)
    I = O.forward_intensity(O.spectrum_from_object(truth), np.ones((16, 16)), geo)
    I = I + 0.01 * np.random.default_rng(seed + 1).standard_normal(I.shape)
    psi = O.spectrum_from_object(smooth_object(geo.N, seed + 2))
    pupil = geo.support * np.exp(0.2j * np.random.default_rng(seed + 3).standard_normal((16, 16)))
    return geo, I, psi, pupil


def test_power_map_reduces_to_eqs_4_and_5():
    """Sec. 6.3: the power map g(x) = x^gamma is the intensity fidelity (Eq. 5) at gamma = 1
    and the amplitude fidelity (Eq. 4) at gamma = 1/2; cost, both gradients and every tile
    must coincide with those forms, which the finite-difference pins check on their own."""
    geo, I, psi, pupil = _fid_problem(41)
    # the maps clamp measurements at 0 (A17) where Eq. 5 does not: compare on I >= 0
    I = np.maximum(I, 0.0)
    for gexp, base in ((1.0, 0), (0.5, 1)):
        a = O.fidelity_cost_grad(psi, pupil, I, geo, O.Options(fidelity=2, g_exponent=gexp), want_tiles=True)
        b = O.fidelity_cost_grad(psi, pupil, I, geo, O.Options(fidelity=base), want_tiles=True)
        assert math.isclose(a[0], b[0], rel_tol=1e-12)
        for x, y in zip(a[1:], b[1:]):
            assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


def test_log_map_is_ln1p_and_its_slope():
    """g(x) = ln(x + 1) of Sec. 6.3 and g' = 1/(x + 1), checked against math.log and a central
    difference of math.log at a few points."""
    opt = O.Options(fidelity=3)
    for x in (0.0, 1e-9, 0.37, 1.0, 12.5):
        # near 0, ln(1 + x) = x - x^2/2 + x^3/3 (math.log(1 + x) would lose the low digits)
        want = x - x * x / 2 + x ** 3 / 3 if x < 1e-3 else math.log(x + 1.0)
        assert math.isclose(float(O.scaling_map(x, opt)), want, rel_tol=1e-14, abs_tol=1e-300)
        a = math.sqrt(x)
        h = 1e-6 * (1.0 + x)
        fd = (math.log(x + h + 1.0) - math.log(x - h + 1.0)) / (2 * h) if x > h else 1.0 / (x + 1.0)
        assert math.isclose(float(O.scaling_map_slope(a, opt)), fd, rel_tol=1e-8)


@pytest.mark.parametrize("variant", [dict(fidelity=2, g_exponent=0.125), dict(fidelity=3)])
def test_zero_gradient_at_the_true_state_for_maps(variant):
    """Noiseless data from the same model: g(|o|^2) - g(I) = 0, so W = 0 for any map."""
    geo, _ = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)
    opt = O.Options(**variant)
    truth = O.spectrum_from_object(smooth_object(geo.N, 23))
    pupil = geo.support.astype(complex)
    I = O.forward_intensity(truth, pupil, geo)
    L, g_psi, g_p, _ = O.fidelity_cost_grad(truth, pupil, I, geo, opt)
    assert math.isclose(L, geo.K * 16 * 16 * opt.tau_fid / 2, rel_tol=1e-6)
    assert np.abs(g_psi).max() < 1e-8 * np.abs(truth).max()
    assert np.abs(g_p).max() < 1e-8


# --------------------------------------------------------------------------- multiplexing (Eq. 1, A18)
def _mux_problem(mux, extra, seed, noise=0.01):
    geo, k_xy = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0, mux=mux, extra_leds=extra)
    truth = smooth_object(geo.N, seed)
    I = O.forward_intensity(O.spectrum_from_object(truth), np.ones((16, 16)), geo)
    I = I + noise * np.random.default_rng(seed + 1).standard_normal(I.shape)
    psi = O.spectrum_from_object(smooth_object(geo.N, seed + 2))
    pupil = geo.support * np.exp(0.2j * np.random.default_rng(seed + 3).standard_normal((16, 16)))
    return geo, k_xy, I, psi, pupil


def test_multiplexed_intensity_is_the_sum_over_its_leds():
    """Eq. 1: image j of an M-LED multiplexed acquisition is the sum of the M sequential images."""
    geo2, k_xy, _, psi, pupil = _mux_problem(2, 1, 51)
    geo1 = O.make_geometry(16, 2, k_xy, na=5.0 / 16, wavelength_um=1.0, pixel_um=1.0)
    I1 = O.forward_intensity(psi, pupil, geo1)
    I2 = O.forward_intensity(psi, pupil, geo2)
    assert I2.shape == (5, 16, 16)
    assert np.allclose(I2, I1[0::2] + I1[1::2], rtol=1e-13, atol=0)
    with pytest.raises(ValueError):
        O.make_geometry(16, 2, k_xy[:9], na=5.0 / 16, wavelength_um=1.0, pixel_um=1.0, mux=2)


@pytest.mark.parametrize("mux,extra,variant", [(2, 1, dict()), (3, 0, dict(fidelity=1)),
                                               (2, 1, dict(fidelity=3, omega_iso=0)),
                                               (5, 1, dict(fidelity=2, g_exponent=0.6))])
def test_multiplexed_gradient_matches_central_differences(mux, extra, variant):
    """Eqs. 9-11 and 18 with M > 1 (the sum over m inside the residual) against central
    differences of the fidelity along 32 seeded complex directions each for Psi and P, h
    scanned over 1e-3 .. 1e-7: agreement to 1e-6."""
    geo, _, I, psi, pupil = _mux_problem(mux, extra, 61)
    opt = O.Options(tau_fid=1e-3, **variant)
    _, g_psi, g_p, _ = O.fidelity_cost_grad(psi, pupil, I, geo, opt)
    rng = np.random.default_rng(62)
    e_psi = fd_worst_error(lambda x: O.fidelity_cost_grad(x, pupil, I, geo, opt)[0], psi, g_psi, rng)
    e_p = fd_worst_error(lambda x: O.fidelity_cost_grad(psi, x, I, geo, opt)[0], pupil, g_p, rng,
                         mask=geo.support)
    print(f"worst of 32 directions: Psi {e_psi:.1e}, P {e_p:.1e}")
    assert e_psi <= FD_TOL and e_p <= FD_TOL


def test_multiplexed_zero_gradient_at_truth_and_order_within_image():
    """Noiseless M = 2 data from the same model give W = 0; reordering the LEDs inside each
    image leaves the cost and g_Psi unchanged and permutes the tiles with the LEDs."""
    geo, k_xy, _, _, _ = _mux_problem(2, 1, 71)
    truth = O.spectrum_from_object(smooth_object(geo.N, 72))
    pupil = geo.support.astype(complex)
    I = O.forward_intensity(truth, pupil, geo)
    L, g_psi, g_p, _ = O.fidelity_cost_grad(truth, pupil, I, geo, O.Options())
    assert math.isclose(L, geo.n_images * 16 * 16 * O.Options().tau_fid / 2, rel_tol=1e-6)
    assert np.abs(g_psi).max() < 1e-9 * np.abs(truth).max() and np.abs(g_p).max() < 1e-9
    _, _, I_n, psi, pupil = _mux_problem(2, 1, 73)
    perm = np.arange(geo.K).reshape(-1, 2)[:, ::-1].ravel()
    geo_p = O.make_geometry(16, 2, k_xy[perm], na=5.0 / 16, wavelength_um=1.0, pixel_um=1.0, mux=2)
    a = O.fidelity_cost_grad(psi, pupil, I_n, geo, O.Options(), want_tiles=True)
    b = O.fidelity_cost_grad(psi, pupil, I_n, geo_p, O.Options(), want_tiles=True)
    assert math.isclose(a[0], b[0], rel_tol=1e-12)
    assert np.linalg.norm(a[1] - b[1]) <= 1e-12 * np.linalg.norm(a[1])
    assert np.linalg.norm(a[3][perm] - b[3]) <= 1e-12 * np.linalg.norm(a[3])


# --------------------------------------------------------------------------- Hessian (A6)
def test_hessian_null_space_and_cross_term():
    N = 24
    yy, xx = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    for f in (3.0 + 0.5 * xx - 0.25 * yy, np.ones((N, N))):
        for c in O.hessian_op(f):
            assert np.abs(c).max() < 1e-12
    dxx, dyy, dxy = O.hessian_op(xx * yy)
    assert np.allclose(dxy[1:-1, 1:-1], math.sqrt(2.0)) and np.abs(dxx).max() == 0 and np.abs(dyy).max() == 0
    dxx, dyy, dxy = O.hessian_op(xx ** 2)
    assert np.allclose(dxx[1:-1, 1:-1], 2.0) and np.abs(dyy).max() == 0 and np.abs(dxy).max() < 1e-12
    # affine amplitude and affine phase (span inside (-pi, pi)): zero gradient, cost = tau/2 per pixel
    amp = 0.5 + 0.01 * xx + 0.005 * yy
    ph = -1.0 + 0.04 * xx + 0.03 * yy
    psi = O.spectrum_from_object(amp * np.exp(1j * ph))
    opt = O.Options()
    L_A, L_P, g = O.hessian_cost_grad(psi, 1.0, 1.0, opt)
    assert math.isclose(L_A, (N - 2) ** 2 * opt.tau_h / 2, rel_tol=1e-6)
    assert math.isclose(L_P, (N - 2) ** 2 * opt.tau_h / 2, rel_tol=1e-6)
    assert np.abs(g).max() < 1e-9


def test_hessian_gradient_wrt_object_matches_differences():
    """Eqs. 13-14 (through F_A^H) for alpha and beta separately against central differences
    of alpha L_A + beta L_Phi along 32 seeded directions, h scanned: agreement to 1e-6."""
    N = 16
    opt = O.Options(tau_h=1e-3)
    obj = smooth_object(N, 31, sigma=2.0)
    psi = O.spectrum_from_object(obj)
    rng = np.random.default_rng(32)
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0)):
        _, _, g = O.hessian_cost_grad(psi, alpha, beta, opt)

        def L(p):
            a, b, _ = O.hessian_cost_grad(p, alpha, beta, opt)
            return alpha * a + beta * b
        err = fd_worst_error(L, psi, g, rng)
        print(f"alpha {alpha} beta {beta}: worst of 32 directions {err:.1e}")
        assert err <= FD_TOL


# --------------------------------------------------------------------------- Eq. 16
def test_alpha_closed_forms():
    n = 20
    assert O.alpha_estimate(np.full((3, n, n), 0.37)) == 0.0
    yy, xx = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    I = np.stack([xx ** 2, xx ** 2])
    # every interior response of [1 2 1]^T (x) [-1 2 -1] to x^2 is -(1+2+1)*2 = -8
    want = 0.2 * math.sqrt(math.pi / 2) * 8.0
    assert math.isclose(O.alpha_estimate(I), want, rel_tol=1e-12)
    assert math.isclose(want, 2.0053026197048, rel_tol=1e-12)
    # amplitude variant (Eq. 17) takes sqrt first: sqrt(x^4) = x^2
    assert math.isclose(O.alpha_estimate(I ** 2, amplitude=True), want, rel_tol=1e-12)
    # the maps of Sec. 6.3 (A17) apply g first: (x^8)^(1/4) = x^2 and ln(e^(x^2/100) - 1 + 1)
    # = x^2 / 100 (kept small so exp stays exact to rounding)
    assert math.isclose(O.alpha_estimate(I ** 4, opt=O.Options(fidelity=2, g_exponent=0.25)), want,
                        rel_tol=1e-12)
    assert math.isclose(O.alpha_estimate(np.expm1(I / 100.0), opt=O.Options(fidelity=3)), want / 100.0,
                        rel_tol=1e-9)
    # negative measurements are clamped before the map: g(max(I, 0)) = 0 for I < 0
    assert O.alpha_estimate(-I, opt=O.Options(fidelity=3)) == 0.0
    assert O.alpha_estimate(-I, opt=O.Options(fidelity=2, g_exponent=0.5)) == 0.0


# --------------------------------------------------------------------------- Eq. 19
def test_adabelief_first_step_closed_form():
    opt = O.Options()
    g = np.array([3 + 4j, -1e-3 + 2e-3j, 0.0])
    x0 = np.array([1 + 1j, 2.0, -3j])
    s0 = 0.7
    x, mu, v, delta, step = O.adabelief(x0, g, np.zeros(3, complex), np.zeros(3), np.full(3, s0 ** 2), 1, opt)
    # t = 1: mu^ = g, v^ = gamma1^2 |g|^2  =>  Delta = (s0 + eta)/(gamma1 |g| + eta) g
    want = (s0 + opt.eta_opt) / (opt.gamma1 * np.abs(g) + opt.eta_opt) * g
    assert np.allclose(step, want, rtol=1e-12, atol=0)
    assert np.allclose(x, x0 - want)
    assert step[2] == 0 and math.isclose(delta[2], opt.gamma1 * s0 ** 2)


def test_adabelief_constant_gradient_closed_form():
    """Constant g: mu_t = (1-g1^t) g so mu^ = g; v_t = (1-g2) g^2 sum_s g2^(t-s) g1^(2s)."""
    opt = O.Options()
    g1, g2 = opt.gamma1, opt.gamma2
    g = np.array([0.3 - 0.4j])
    x = np.zeros(1, complex)
    mu = np.zeros(1, complex)
    v = np.zeros(1)
    delta = np.ones(1)
    for t in range(1, 8):
        x, mu, v, delta, _ = O.adabelief(x, g, mu, v, delta, t, opt)
        assert np.allclose(mu, (1 - g1 ** t) * g, rtol=1e-13)
        vt = (1 - g2) * abs(g[0]) ** 2 * sum(g2 ** (t - s) * g1 ** (2 * s) for s in range(1, t + 1))
        assert math.isclose(v[0], vt, rel_tol=1e-12)


# --------------------------------------------------------------------------- pupil update (A15)
def _gauss3_by_hand(p):
    """3 x 3 Gaussian of sigma 1 px (weights e^{-(dy^2 + dx^2)/2}, normalised to sum 1) applied
    with zero padding, one output pixel at a time."""
    n0, n1 = p.shape
    w = {(dy, dx): math.exp(-0.5 * (dy * dy + dx * dx)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)}
    z = sum(w.values())
    out = np.zeros_like(p)
    for y in range(n0):
        for x in range(n1):
            acc = 0j
            for (dy, dx), wt in w.items():
                if 0 <= y + dy < n0 and 0 <= x + dx < n1:
                    acc += wt / z * p[y + dy, x + dx]
            out[y, x] = acc
    return out


def _pupil_problem():
    geo, k_xy = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)
    truth = smooth_object(geo.N, 91)
    I = O.forward_intensity(O.spectrum_from_object(truth), np.ones((16, 16)), geo)
    I = I + 0.01 * np.random.default_rng(92).standard_normal(I.shape)
    opt = O.Options()
    st = O.init_state(I, geo, k_xy, opt)
    # a pupil that varies across the support, so that the filter also changes it inside S
    st.pupil = geo.support * (1.0 + 0.2 * np.random.default_rng(93).standard_normal((16, 16))) * np.exp(
        0.3j * np.random.default_rng(94).standard_normal((16, 16)))
    return geo, I, opt, st


def test_pupil_update_composition_first_iteration():
    """Note under Algorithm 1 (reading A15): P^1 = mask_S o (G3 (x) P^0 - Delta_P), where Delta_P
    is Eq. 19's first step at the gradient of Eq. 18 taken at the unfiltered P^0:
    Delta = (s0 + eta) / (gamma1 |g| + eta) g (mu^ = g, v^ = gamma1^2 |g|^2 at t = 1).  The filter
    is summed by hand here.  The three other readings (step before the filter, no mask, no
    filter) must give a different pupil, so a swapped order or a dropped mask fails this pin."""
    geo, I, opt, st = _pupil_problem()
    _, _, g_p, _ = O.fidelity_cost_grad(st.psi, st.pupil, I, geo, opt)
    assert np.abs(g_p).max() > 0 and np.all(g_p[~geo.support] == 0)
    new, _, _ = O.iteration(st, I, geo, opt)
    g1, g2, eta, s0 = opt.gamma1, opt.gamma2, opt.eta_opt, opt.s0_pupil
    step = (s0 + eta) / (g1 * np.abs(g_p) + eta) * g_p
    filtered = _gauss3_by_hand(st.pupil)
    want = geo.support * (filtered - step)
    scale = np.abs(want).max()
    assert np.abs(new.pupil - want).max() <= 1e-13 * scale
    # the optimiser state of P after its first step (Eq. 19 at t = 1 from mu = v = 0, delta = s0^2)
    assert np.allclose(new.mu_p, (1 - g1) * g_p, rtol=1e-13, atol=0)
    assert np.allclose(new.v_p, (1 - g2) * g1 ** 2 * np.abs(g_p) ** 2, rtol=1e-12, atol=0)
    assert np.allclose(new.delta_p, g1 * s0 ** 2 + (1 - g1) * np.abs(step) ** 2, rtol=1e-13, atol=0)
    # the other compositions are distinguishable from the reading
    for alt in (geo.support * _gauss3_by_hand(st.pupil - step),   # step, then filter, then mask
                filtered - step,                                  # no mask
                geo.support * (st.pupil - step)):                 # no filter
        assert np.abs(alt - want).max() > 1e-3 * scale


def test_update_norms_first_iteration():
    """The norms of a Psi update (the FP64 norms of the cost row): ||g|| of the full gradient
    g = dL/dconj(Psi) of Eq. 8 (Eq. 9 plus the Hessian terms, each pinned on its own above) and
    ||Delta Psi||, which at t = 1 has the closed form of Eq. 19's first step,
    sqrt(sum ((s0 + eta) |g| / (gamma1 |g| + eta))^2), and equals the distance between the states
    the iteration returns.  Using the fidelity gradient alone, the moment instead of the step, or
    a missing square root fails one of these."""
    geo, I, opt, st = _pupil_problem()
    _, g_fid, _, _ = O.fidelity_cost_grad(st.psi, st.pupil, I, geo, opt)
    _, _, g_h = O.hessian_cost_grad(st.psi, st.alpha, st.beta, opt)
    g = g_fid + g_h
    assert np.abs(g_h).max() > 1e-3 * np.abs(g_fid).max()
    norms = []
    new, _, _ = O.iteration(st, I, geo, opt, norms=norms)
    assert len(norms) == 1
    ng, nd = norms[0]
    want_g = math.sqrt(sum(abs(z) ** 2 for z in g.ravel()))
    g1, eta, s0 = opt.gamma1, opt.eta_opt, opt.s0_psi
    want_d = math.sqrt(sum(((s0 + eta) * abs(z) / (g1 * abs(z) + eta)) ** 2 for z in g.ravel()))
    assert math.isclose(ng, want_g, rel_tol=1e-12)
    assert math.isclose(nd, want_d, rel_tol=1e-12)
    assert math.isclose(nd, float(np.linalg.norm(new.psi - st.psi)), rel_tol=1e-10)
    assert not math.isclose(ng, float(np.linalg.norm(g_fid)), rel_tol=1e-6)


def test_pupil_update_without_filter_and_fixed_pupil():
    """pupil_filter = 0 drops the Gaussian only: P^1 = mask_S o (P^0 - Delta_P); learn_pupil = 0
    leaves P and its optimiser state untouched while Psi still moves."""
    geo, I, _, st = _pupil_problem()
    opt = O.Options(pupil_filter=0)
    _, _, g_p, _ = O.fidelity_cost_grad(st.psi, st.pupil, I, geo, opt)
    new, _, _ = O.iteration(st, I, geo, opt)
    step = (opt.s0_pupil + opt.eta_opt) / (opt.gamma1 * np.abs(g_p) + opt.eta_opt) * g_p
    want = geo.support * (st.pupil - step)
    assert np.abs(new.pupil - want).max() <= 1e-13 * np.abs(want).max()
    fixed, _, _ = O.iteration(st, I, geo, O.Options(learn_pupil=0))
    assert np.array_equal(fixed.pupil, st.pupil) and np.array_equal(fixed.delta_p, st.delta_p)
    assert not np.any(fixed.mu_p) and not np.array_equal(fixed.psi, st.psi)


# --------------------------------------------------------------------------- Algorithm 1
def test_initial_state_reproduces_centre_image():
    """Psi0 built from the centre-LED image reproduces that image's amplitude (Nyquist aside)."""
    geo, k_xy = tiny_problem(n=16, u=2, grid=3, step=4, na_px=8.0)
    truth = O.spectrum_from_object(smooth_object(geo.N, 41, sigma=2.0))
    I = O.forward_intensity(truth, geo.support.astype(complex), geo)
    st = O.init_state(I, geo, k_xy, O.Options(alpha=0.0, beta=0.0))
    assert O.centre_led(k_xy) == 4
    o = O.forward_field(st.psi, np.ones((16, 16)), geo, 4)
    assert np.abs(o.imag).max() < 1e-12
    obj0 = O.object_from_spectrum(st.psi)        # Nyquist row/column zeroed => real O0
    assert np.abs(obj0.imag).max() < 1e-12 * np.abs(obj0).max()
    assert np.allclose(np.abs(o), np.sqrt(I[4]), atol=0.05)
    assert st.t == 0 and np.all(st.delta_psi == 1.0) and np.all(st.delta_p == 1e-4)


def test_noiseless_convergence():
    """learn_pupil=0, alpha=beta=0, noiseless data: the fidelity drops by > 3 orders.
    The rate is parity unpinned against the paper (which only says 'within 20 iterations')."""
    geo, k_xy = tiny_problem(n=16, u=4, grid=5, step=3, na_px=4.5)
    truth = O.spectrum_from_object(smooth_object(geo.N, 51, sigma=3.0))
    I = O.forward_intensity(truth, geo.support.astype(complex), geo)
    opt = O.Options(learn_pupil=0, alpha=0.0, beta=0.0, tau_fid=1e-9)
    st = O.init_state(I, geo, k_xy, opt)
    st, costs = O.run(st, I, geo, opt, 150)
    floor = geo.K * 16 * 16 * opt.tau_fid / 2
    assert (costs[-1, 0] - floor) < 1e-3 * (costs[0, 0] - floor), costs[[0, -1], 0]


def test_hessian_fills_spectrum_beyond_passband():
    """Sec. 4.2: with the Hessian term the recovered spectrum is nonzero beyond the
    region the LEDs cover; the initial spectrum is zero there."""
    geo, k_xy = tiny_problem(n=16, u=4, grid=3, step=3, na_px=4.0)
    truth = O.spectrum_from_object(smooth_object(geo.N, 61, sigma=3.0))
    I = O.forward_intensity(truth, geo.support.astype(complex), geo)
    st = O.init_state(I, geo, k_xy, O.Options(alpha=0.05, beta=0.05))
    corner = (slice(0, 8), slice(0, 8))
    assert np.abs(st.psi[corner]).max() == 0
    st2, _, _ = O.iteration(st, I, geo, O.Options(alpha=0.05, beta=0.05))
    assert np.abs(st2.psi[corner]).min() > 0


def test_initial_phase_is_ill_conditioned():
    """The initial object O0 is real (phase exactly 0), so the phase term of Eq. 14 at the
    first iteration normalises pure rounding noise: noise of FP32 size (1e-7 relative) in O
    changes the first step's phase-Hessian cost by a large factor.  This is a property of the
    method at that state, not of an implementation; it bounds FP32-vs-FP64 agreement of any
    run that starts from the initial state."""
    import oracle.elfpie_oracle as OE
    geo, k_xy = tiny_problem(n=32, u=4, grid=3, step=5, na_px=6.0)
    truth = O.spectrum_from_object(smooth_object(geo.N, 71, sigma=4.0))
    I = O.forward_intensity(truth, geo.support.astype(complex), geo)
    I = I + 1e-3 * np.random.default_rng(72).standard_normal(I.shape)
    opt = O.Options()
    st = O.init_state(I, geo, k_xy, opt)
    _, c_ref = O.run(st, I, geo, opt, 2)
    orig = OE.object_from_spectrum
    rng = np.random.default_rng(73)

    def noisy(psi):
        o = orig(psi)
        return o + 1e-7 * np.abs(o).mean() * (rng.standard_normal(o.shape) + 1j * rng.standard_normal(o.shape))
    try:
        OE.object_from_spectrum = noisy
        _, c_pert = O.run(st, I, geo, opt, 2)
    finally:
        OE.object_from_spectrum = orig
    # iteration 0 costs agree; the phase cost after one step does not
    assert abs(c_pert[0, 2] - c_ref[0, 2]) < 1e-3 * c_ref[0, 2]
    assert abs(c_pert[1, 2] - c_ref[1, 2]) > 0.1 * c_ref[1, 2]


# --------------------------------------------------------------------------- Sec. 4.1 evaluation
def test_periodic_gaussian_kernel_and_circular_convolution():
    """G of Eq. 20 (A19): unit sum, exp(-2/w^2) between neighbours; the direct circular sum (A20)
    of a shifted delta is the shifted kernel, and it equals the convolution theorem's product."""
    n, w = 12, 3.0
    g = O.gaussian_kernel_periodic(n, w)
    assert math.isclose(g.sum(), 1.0, rel_tol=1e-14)
    assert math.isclose(g[0, 1] / g[0, 0], math.exp(-2.0 / w ** 2), rel_tol=1e-14)
    assert math.isclose(g[1, 1] / g[0, 0], math.exp(-4.0 / w ** 2), rel_tol=1e-14)
    assert np.allclose(g, g.T) and np.allclose(g[1:], g[1:][::-1])
    delta = np.zeros((n, n))
    delta[3, 5] = 1.0
    assert np.allclose(O.circular_convolve(delta, g), np.roll(np.roll(g, 3, axis=0), 5, axis=1), atol=1e-16)
    f = np.random.default_rng(81).standard_normal((n, n))
    via_fft = np.real(np.fft.ifft2(np.fft.fft2(f) * np.fft.fft2(g)))
    assert np.allclose(O.circular_convolve(f, g), via_fft, atol=1e-13)
    h = np.random.default_rng(86).standard_normal((n, n))  # not symmetric: orientation matters
    assert np.allclose(O.circular_convolve(f, h), np.real(np.fft.ifft2(np.fft.fft2(f) * np.fft.fft2(h))), atol=1e-12)


def test_illumination_pattern_spans_one_minus_c_to_one():
    zeta = np.random.default_rng(82).standard_normal((16, 16))
    L = O.illumination_pattern(zeta, 0.3, 4.0)
    assert math.isclose(L.min(), 0.7, rel_tol=1e-14) and math.isclose(L.max(), 1.0, rel_tol=1e-14)
    assert np.all(O.illumination_pattern(np.full((8, 8), 2.5), 0.3, 4.0) == 0.7)


def test_degrade_terms():
    """Eqs. 2 / 20: with c = 0 the output minus the clean image is Omega + a xi exactly; the
    salt & pepper rule maps u < d/2 to 0 and d/2 <= u < d to 1 and leaves the rest."""
    g = np.random.default_rng(83)
    I0 = g.uniform(0.1, 1.0, (3, 8, 8))
    xi = g.standard_normal(I0.shape)
    bg = np.array([0.01, 0.02, 0.03])
    out = O.degrade(I0, background=bg, gauss_a=0.05, xi=xi)
    assert np.allclose(out - I0, bg[:, None, None] + 0.05 * xi, atol=1e-15)
    u = np.array([0.0, 0.049, 0.05, 0.0999, 0.1, 0.7]).reshape(1, 1, 6)
    out = O.degrade(np.full((1, 1, 6), 0.4), snp_density=0.1, u_snp=u)
    assert out.ravel().tolist() == [0.0, 0.0, 1.0, 1.0, 0.4, 0.4]
    zeta = g.standard_normal(I0.shape)
    out = O.degrade(I0, c=0.4, waist_px=3.0, zeta=zeta)
    ratio = out / I0
    assert np.allclose(ratio.min(axis=(1, 2)), 0.6) and np.allclose(ratio.max(axis=(1, 2)), 1.0)


def test_noise_level_and_darkfield_selection():
    """Eq. 21 on a hand example (10 % on the one dark image, bright images ignored) and the
    dark-field rule |c_n| dk > NA / lambda with all LEDs of an image dark."""
    I_sim = np.full((3, 4, 4), 2.0)
    I_noi = I_sim.copy()
    I_noi[1] += 0.2
    I_noi[0] += 5.0
    assert math.isclose(O.noise_level(I_sim, I_noi, [False, True, False]), 10.0, rel_tol=1e-14)
    assert math.isclose(O.noise_level(I_sim, I_noi, [True, True, False]), (250.0 + 10.0) / 2, rel_tol=1e-14)
    geo, _ = tiny_problem(n=16, u=2, grid=3, step=4, na_px=5.0)  # offsets 0, +-4 px; pupil radius 5 px
    # the diagonal LEDs sit at 4 sqrt(2) = 5.66 px > 5: dark; the edge LEDs at 4 px: bright
    assert O.darkfield_images(geo, 5.0 / 16, 1.0).tolist() == [True, False, True, False, False, False, True,
                                                               False, True]
    geo, _ = tiny_problem(n=16, u=4, grid=3, step=6, na_px=5.0)  # +-6 px: all but the centre are dark
    dark = O.darkfield_images(geo, 5.0 / 16, 1.0)
    assert dark.tolist() == [True] * 4 + [False] + [True] * 4
    geo3 = O.make_geometry(16, 4, np.asarray(_grid_k(3, 6, 16)), na=5.0 / 16, wavelength_um=1.0, pixel_um=1.0,
                           mux=3)
    assert O.darkfield_images(geo3, 5.0 / 16, 1.0).tolist() == [True, False, True]


def _grid_k(grid, step, n):
    c = (np.arange(grid) - (grid - 1) // 2) * step
    cy, cx = np.meshgrid(c, c, indexing="ij")
    return np.stack([cx.ravel() / n, cy.ravel() / n], axis=1)


def test_lsnr_is_the_maximum_over_b():
    """Eq. 22: the closed-form b attains the maximum of the printed expression (checked on a
    fine grid of b), a hand example, and invariance to a constant added to the estimate."""
    g = np.random.default_rng(84)
    truth = g.uniform(0.1, 1.0, 50)
    rec = truth + 0.05 * g.standard_normal(50) + 0.3
    val = O.lsnr(rec, truth)
    bs = np.linspace(-1.0, 1.0, 200001)
    d = truth[None, :] - rec[None, :] - bs[:, None]
    brute = np.max(10 * np.log10(np.sum(truth ** 2) / np.sum(d ** 2, axis=1)))
    assert val >= brute - 1e-9 and val - brute < 1e-6
    assert math.isclose(O.lsnr(rec + 7.0, truth), val, rel_tol=1e-12)
    # truth (1, 3), rec (0, 0): b = 2, residual (-1, 1), 10 log10(10 / 2)
    assert math.isclose(O.lsnr([0.0, 0.0], [1.0, 3.0]), 10 * math.log10(5.0), rel_tol=1e-14)


def test_object_quality_ignores_the_global_phase():
    g = np.random.default_rng(85)
    truth = g.uniform(0.2, 1.0, (8, 8)) * np.exp(1j * g.uniform(-1.0, 1.0, (8, 8)))
    rec = truth + 0.01 * (g.standard_normal((8, 8)) + 1j * g.standard_normal((8, 8)))
    a0, p0 = O.object_quality(rec, truth)
    a1, p1 = O.object_quality(rec * np.exp(0.9j), truth)
    assert math.isclose(a0, a1, rel_tol=1e-12) and math.isclose(p0, p1, rel_tol=1e-9)
    assert 25.0 < a0 < 60.0 and 15.0 < p0 < 60.0
    # phases spanning (-3, 3): a global phase left in place would wrap part of the map
    truth = g.uniform(0.2, 1.0, (8, 8)) * np.exp(1j * g.uniform(-3.0, 3.0, (8, 8)))
    rec = truth * np.exp(0.9j) * (1.0 + 1e-3 * g.standard_normal((8, 8)))
    assert O.object_quality(rec, truth)[1] > 40.0


def test_normaliser_at_tau_zero_is_the_l1_subgradient_zero_at_the_origin():
    """tau = 0 is the paper's plain L1 with its gradient taken as 0 at the origin (Sec. 3.3):
    omega = x / |x| away from 0 and exactly 0 there, the cost |x|; no NaN anywhere."""
    x = np.array([3.0, 0.0, -2.0, 0.0])
    y = np.array([4.0, 0.0, 0.0, -1e-300])
    cost, (wx, wy) = O.huber([x, y], 0.0, 1)
    assert np.allclose(cost, np.hypot(x, y)) and np.all(np.isfinite(wx)) and np.all(np.isfinite(wy))
    assert wx.tolist()[:3] == [0.6, 0.0, -1.0] and wy.tolist()[:3] == [0.8, 0.0, 0.0]
    cost, (wx, wy) = O.huber([x, y], 0.0, 0)
    assert np.allclose(cost, np.abs(x) + np.abs(y))
    assert wx.tolist() == [1.0, 0.0, -1.0, 0.0] and wy.tolist() == [1.0, 0.0, 0.0, -1.0]
