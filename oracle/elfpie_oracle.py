"""Plain, slow, FP64 reference of one Elfpie iteration (arXiv 2209.14671).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline legs, never by the CUDA product path.

Everything is complex128 / float64 NumPy, one operation per line, in the order of
Algorithm 1 (Sec. 3.4).  The paper leaves several points silent or garbled; the
readings taken here are labelled A1..A20 and listed with their reasons in the
design notes of the repository.  In short:

* A1  transforms: Psi = fftshift(DFT_N(O)), O = IDFT_N(ifftshift(Psi)) (IDFT
      carries 1/A); o_n = u^-2 IDFT_n(ifftshift(P o C_n Psi)).  Sec. 3.1, Eqs. 1, 6.
* A3  LED offset c_n = round-half-away-from-zero(k_n / dk), dk = 1/(n dx).
* A4  pupil support S = {|j - n/2|^2 dk^2 <= (NA/lambda)^2}.
* A5  nabla = forward differences with a Neumann (zero) last row/column.
* A6  H = (Dxx, Dyy, sqrt2 Dxy) on the valid interior [1, N-2]^2.
* A7  the L1 "gradient 0 at the origin" rule (Sec. 3.3) is a Huber smoothing:
      phi(x) = |x| for |x| >= tau, |x|^2/(2 tau) + tau/2 below; tau = 0 is the
      paper literally, with omega = 0 where the feature is exactly 0.
* A8  Eq. 11's residual is model minus measured in the intensity domain.
* A9  initial state: Psi0 from the centre-LED image, mu = v = 0, delta = s0^2.
* A10 alpha (Eq. 16): 'valid' 3x3 correlation, mean over the (n-2)^2 interior.
* A11 every gradient is the true dL/d(conj z) (Eq. 10's missing 1/2 restored).
* A12 phase = atan2 without unwrapping.  A13 eta_H = 1e-12.  A14 eta_opt = 1e-8.
* A15 pupil: P~ = G3 (x) P, P_new = mask o (P~ - Delta_P), gradient at P^t.
* A16 s0_P = 1e-2.
* A17 gamma / log fidelity (Sec. 6.3): g(x) = x^gamma or ln(x + 1) replaces
      the identity (Eq. 5) or sqrt (Eq. 4) map of Eq. 3; measured intensities
      are clamped at 0 before the map, and the slope g'(|o|^2) of the power map
      takes |o| floored at eta_H, so gamma = 1/2 is exactly the amplitude form.
      Eqs. 16-17 take g(max(I, 0)) for these maps.
* A18 multiplexing (Eq. 1 with M > 1): LEDs in the caller's order, image j is
      lit by LEDs jM .. jM+M-1 (K a multiple of M); the residual of image j
      uses sum_m |o_{j,m}|^2; Psi0 comes from the image holding the centre LED.
* A19 Eq. 20's G (x) zeta: G = exp(-2 r^2 / w^2), w the "half-waist" read as the
      1/e^2 radius; the blurred field min-max normalised to [0, 1] per image so
      that c sets the illumination range [1 - c, 1].
* A20 that convolution is circular on the n x n image grid.

Parity status: every function below is pinned by ``tests/test_oracle_pins.py``
(brute-force DFT, Parseval, adjoint identities, central differences along 32
seeded directions with a scanned step, affine null space of H, closed forms for
alpha and the first AdaBelief step, the pupil update of ``iteration`` against a
hand-summed filter and the closed-form first step, the update norms against the first step's
closed form and the returned states, noiseless convergence).  The reconstruction-quality numbers of the paper's Tables 2-4 are
parity unpinned (their images and comparison codes are not available).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Options", "Geometry", "State", "round_half_away", "make_geometry",
    "crop", "crop_adjoint", "forward_field", "forward_intensity",
    "grad_op", "grad_adj", "huber", "hessian_op", "hessian_adj",
    "fidelity_cost_grad", "object_from_spectrum", "spectrum_from_object",
    "hessian_cost_grad", "adabelief", "update_norms", "gauss3", "filter3", "alpha_estimate",
    "scaling_map", "scaling_map_slope",
    "init_state", "iteration", "run", "total_cost", "centre_led",
    "LAPLACE_KERNEL", "gaussian_kernel_periodic", "circular_convolve", "illumination_pattern",
    "degrade", "darkfield_images", "noise_level", "lsnr", "object_quality",
]


# ----------------------------------------------------------------------------
# options and geometry
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    """Hyper-parameters of Sec. 6.2 and the smoothing constants of the readings.

    fidelity: 0 = intensity (Eq. 5, default), 1 = amplitude (Eq. 4),
              2 = power map g(x) = x^g_exponent, 3 = log map g(x) = ln(x + 1)
              (Sec. 6.3, A17).
    g_exponent: the gamma of the power map (fidelity 2).
    omega_iso: 1 = isotropic normaliser (Eq. 12 first case), 0 = anisotropic.
    alpha/beta < 0 select the automatic estimate of Eqs. 16-17.
    gamma1, gamma2: the r1, r2 of Sec. 6.2 (0.9 / 0.999).
    s0_psi, s0_pupil: initial step sqrt(delta^0) of Eq. 19 for Psi and P.
    """
    fidelity: int = 0
    omega_iso: int = 1
    learn_pupil: int = 1
    pupil_filter: int = 1
    alpha: float = -1.0
    beta: float = -1.0
    gamma1: float = 0.9
    gamma2: float = 0.999
    s0_psi: float = 1.0
    s0_pupil: float = 1e-2
    eta_opt: float = 1e-8
    eta_h: float = 1e-12
    tau_fid: float = 1e-6
    tau_h: float = 1e-4
    g_exponent: float = 1.0


@dataclasses.dataclass
class Geometry:
    n: int                 # low-res side, B = n*n
    u: int                 # upsampling, N = u*n
    N: int                 # high-res side, A = N*N
    dk: float              # spectral pixel (cycles/um), same on both grids
    offsets: np.ndarray    # int64 [K, 2] = (c_y, c_x) in spectral pixels (A3)
    origins: np.ndarray    # int64 [K, 2] = crop window top-left (row, col) in Psi
    support: np.ndarray    # bool [n, n] pupil support S (A4)
    mux: int = 1           # M: LEDs lit together per measured image (Eq. 1, A18)

    @property
    def K(self) -> int:
        return int(self.offsets.shape[0])

    @property
    def n_images(self) -> int:
        """Number of measured images, K / M."""
        return self.K // self.mux


def round_half_away(x):
    """Round to nearest, halves away from zero (A3)."""
    x = np.asarray(x, dtype=np.float64)
    return (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)


def make_geometry(n, u, k_xy, na, wavelength_um, pixel_um, mux=1) -> Geometry:
    """Crop windows M_n and pupil support of the forward model (Sec. 3.1, Eq. 1).

    k_xy: [K, 2] illumination spatial frequency (kx, ky) in cycles/um.
    pixel_um: low-res pixel size at the sample plane.
    mux: M, the LEDs lit together for one image (A18: image j = LEDs jM .. jM+M-1).
    The spectral spacing is dk = 1/(n*pixel_um) on both grids (N*pixel_um/u = n*pixel_um).
    """
    n = int(n)
    u = int(u)
    N = n * u
    dk = 1.0 / (n * float(pixel_um))
    k_xy = np.asarray(k_xy, dtype=np.float64).reshape(-1, 2)
    cy = round_half_away(k_xy[:, 1] / dk)
    cx = round_half_away(k_xy[:, 0] / dk)
    offsets = np.stack([cy, cx], axis=1)
    origins = offsets + (N // 2 - n // 2)
    if np.any(origins < 0) or np.any(origins + n > N):
        raise ValueError("an LED crop window falls outside the high-res spectrum")
    j = np.arange(n) - n // 2
    rho2 = (j[None, :] ** 2 + j[:, None] ** 2) * dk * dk
    support = rho2 <= (float(na) / float(wavelength_um)) ** 2
    mux = int(mux)
    if mux < 1 or k_xy.shape[0] % mux:
        raise ValueError("the LED count must be a positive multiple of mux")
    return Geometry(n=n, u=u, N=N, dk=dk, offsets=offsets, origins=origins, support=support, mux=mux)


# ----------------------------------------------------------------------------
# forward model (Sec. 3.1, Eq. 1)
# ----------------------------------------------------------------------------
def crop(psi, geo: Geometry, led: int):
    """M_n Psi: the n x n window of the centred spectrum for LED ``led``."""
    oy, ox = geo.origins[led]
    return psi[oy:oy + geo.n, ox:ox + geo.n]


def crop_adjoint(tile, geo: Geometry, led: int):
    """M_n^T: put an n x n tile back at its place in an N x N zero spectrum."""
    out = np.zeros((geo.N, geo.N), dtype=np.complex128)
    oy, ox = geo.origins[led]
    out[oy:oy + geo.n, ox:ox + geo.n] = tile
    return out


def forward_field(psi, pupil, geo: Geometry, led: int):
    """o_n = F_B P M_n Psi (Eq. 1, A1): u^-2 * IDFT_n(ifftshift(P o crop))."""
    p = pupil * geo.support
    t = p * crop(psi, geo, led)
    return np.fft.ifft2(np.fft.ifftshift(t)) / (geo.u * geo.u)


def forward_intensity(psi, pupil, geo: Geometry):
    """Predicted low-res intensities of Eq. 1, float64 [K/M, n, n]: image j is
    sum_m |o_{j,m}|^2 over its M LEDs (|o_n|^2 per LED when M = 1)."""
    out = np.zeros((geo.n_images, geo.n, geo.n), dtype=np.float64)
    for k in range(geo.K):
        out[k // geo.mux] += np.abs(forward_field(psi, pupil, geo, k)) ** 2
    return out


# ----------------------------------------------------------------------------
# first-order difference operator (A5) and its adjoint
# ----------------------------------------------------------------------------
def grad_op(r):
    """nabla r = (nabla_x r, nabla_y r): forward differences, zero on the last column/row."""
    gx = np.zeros_like(r)
    gy = np.zeros_like(r)
    gx[:, :-1] = r[:, 1:] - r[:, :-1]
    gy[:-1, :] = r[1:, :] - r[:-1, :]
    return gx, gy


def grad_adj(px, py):
    """nabla^T (px, py): the exact transpose of grad_op."""
    out = np.zeros_like(px)
    out[:, 1:] += px[:, :-1]
    out[:, :-1] -= px[:, :-1]
    out[1:, :] += py[:-1, :]
    out[:-1, :] -= py[:-1, :]
    return out


# ----------------------------------------------------------------------------
# the normaliser omega of Eq. 12 under the smoothing reading A7
# ----------------------------------------------------------------------------
def huber(comps, tau, iso):
    """Per-pixel cost phi_tau and its gradient omega (Eq. 12 with A7).

    comps: list of equally shaped arrays (the components of the feature vector).
    iso=1: phi = ||x||_2 if ||x|| >= tau else ||x||^2/(2 tau) + tau/2,
           omega = x / max(||x||, tau).
    iso=0: the same rule on each component separately (omega_i = x_i/max(|x_i|,tau)).
    With tau = 0 (the paper literally) omega is 0 where the norm is 0: the L1 gradient
    at the origin is taken as zero (Sec. 3.3).
    Returns (cost array, list of omega arrays).
    """
    def ratio(c, den):
        return np.divide(c, den, out=np.zeros_like(c), where=den > 0)

    def smooth(a):
        if tau <= 0:
            return a
        return np.where(a >= tau, a, a * a / (2.0 * tau) + tau / 2.0)

    if iso:
        norm = np.sqrt(sum(c * c for c in comps))
        den = np.maximum(norm, tau)
        return smooth(norm), [ratio(c, den) for c in comps]
    cost = np.zeros_like(comps[0])
    omegas = []
    for c in comps:
        a = np.abs(c)
        cost = cost + smooth(a)
        omegas.append(ratio(c, np.maximum(a, tau)))
    return cost, omegas


# ----------------------------------------------------------------------------
# second-order operator H (A6) and its adjoint
# ----------------------------------------------------------------------------
def hessian_op(f):
    """H f = (Dxx, Dyy, sqrt(2) Dxy) on the interior (1..N-2)^2, zero elsewhere (Sec. 3.2)."""
    dxx = np.zeros_like(f)
    dyy = np.zeros_like(f)
    dxy = np.zeros_like(f)
    c = f[1:-1, 1:-1]
    dxx[1:-1, 1:-1] = f[1:-1, :-2] - 2.0 * c + f[1:-1, 2:]
    dyy[1:-1, 1:-1] = f[:-2, 1:-1] - 2.0 * c + f[2:, 1:-1]
    dxy[1:-1, 1:-1] = (f[2:, 2:] - f[2:, :-2] - f[:-2, 2:] + f[:-2, :-2]) / 4.0
    return dxx, dyy, math.sqrt(2.0) * dxy


def hessian_adj(wxx, wyy, wxy):
    """H^T (wxx, wyy, wxy): exact transpose of hessian_op (inputs live on the interior)."""
    out = np.zeros_like(wxx)
    a = wxx[1:-1, 1:-1]
    out[1:-1, :-2] += a
    out[1:-1, 1:-1] -= 2.0 * a
    out[1:-1, 2:] += a
    b = wyy[1:-1, 1:-1]
    out[:-2, 1:-1] += b
    out[1:-1, 1:-1] -= 2.0 * b
    out[2:, 1:-1] += b
    c = math.sqrt(2.0) * wxy[1:-1, 1:-1] / 4.0
    out[2:, 2:] += c
    out[2:, :-2] -= c
    out[:-2, 2:] -= c
    out[:-2, :-2] += c
    return out


# ----------------------------------------------------------------------------
# the pixel-wise scaling g of Eq. 3 beyond Eqs. 4-5 (Sec. 6.3, A17)
# ----------------------------------------------------------------------------
def scaling_map(x, opt: Options):
    """g(x) for a non-negative intensity x: x^gamma (fidelity 2) or ln(x + 1)
    (fidelity 3), the gamma-correction and logarithmic maps of Sec. 6.3."""
    x = np.asarray(x, dtype=np.float64)
    if opt.fidelity == 2:
        return x ** opt.g_exponent
    if opt.fidelity == 3:
        return np.log1p(x)
    raise ValueError("scaling_map is defined for fidelity 2 and 3")


def scaling_map_slope(amp, opt: Options):
    """g'(|o|^2) as a function of amp = |o|: gamma * max(|o|, eta_H)^(2 gamma - 2)
    for the power map (the floor of Eq. 10's 1/|o| carried over, A13/A17), and
    1 / (|o|^2 + 1) for the log map."""
    amp = np.asarray(amp, dtype=np.float64)
    if opt.fidelity == 2:
        return opt.g_exponent * np.maximum(amp, opt.eta_h) ** (2.0 * opt.g_exponent - 2.0)
    if opt.fidelity == 3:
        return 1.0 / (amp * amp + 1.0)
    raise ValueError("scaling_map_slope is defined for fidelity 2 and 3")


# ----------------------------------------------------------------------------
# data fidelity (Eqs. 4-5) and its Wirtinger gradients (Eqs. 9-11, 18)
# ----------------------------------------------------------------------------
def fidelity_cost_grad(psi, pupil, I, geo: Geometry, opt: Options, want_tiles=False):
    """L_fid and its gradients with respect to conj(Psi) and conj(P).

    For each measured image j (Algorithm 1, inner loops), lit by the LEDs
    m = jM .. jM+M-1 (A18; M = 1 is sequential FPM):
      o_m = forward_field                                  (Eq. 1)
      s_j = sum_m |o_m|^2                                  (Eq. 1)
      r_j = s_j - I_j                (intensity, Eq. 5, A8)
          = sqrt(s_j) - sqrt(max(I_j,0)) (amplitude, Eq. 4)
          = g(s_j) - g(max(I_j,0))   (power / log map, Sec. 6.3, A17)
      d = nabla r_j; (phi, omega) = huber(d)               (Eq. 12, A7)
      W_m = o_m o nabla^T omega                            (intensity, Eq. 11)
          = o_m / (2 max(sqrt(s_j), eta_H)) o nabla^T omega (amplitude, Eq. 10, A11)
          = g'(s_j) o_m o nabla^T omega                    (power / log map: chain rule
            of Eq. 3, d s_j / d conj(o_m) = o_m)
      G_m = u^-2 n^-2 fftshift(DFT_n(W_m))                 (F_B^H of Eq. 9)
    then (sums in ascending LED order)
      g_Psi = sum_m M_m^T (conj(P) o G_m)                  (Eq. 9)
      g_P   = sum_m conj(M_m Psi) o G_m, masked to S       (Eq. 18)
    I holds the K/M measured images.
    Returns (L_fid, g_psi [N,N], g_pupil [n,n], tiles [K,n,n] or None).
    """
    n, u, M = geo.n, geo.u, geo.mux
    mask = geo.support
    p_eff = pupil * mask
    g_psi = np.zeros((geo.N, geo.N), dtype=np.complex128)
    g_p = np.zeros((n, n), dtype=np.complex128)
    tiles = np.zeros((geo.K, n, n), dtype=np.complex128) if want_tiles else None
    cost = 0.0
    for j in range(geo.n_images):
        leds = range(j * M, (j + 1) * M)
        fields = [forward_field(psi, pupil, geo, k) for k in leds]
        s = np.zeros((n, n))
        for o in fields:
            s += np.abs(o) ** 2
        if opt.fidelity == 0:
            r = s - I[j]
        elif opt.fidelity == 1:
            r = np.sqrt(s) - np.sqrt(np.maximum(I[j], 0.0))
        else:
            r = scaling_map(s, opt) - scaling_map(np.maximum(I[j], 0.0), opt)
        dx, dy = grad_op(r)
        phi, (wx, wy) = huber([dx, dy], opt.tau_fid, opt.omega_iso)
        cost += float(np.sum(phi))
        w = grad_adj(wx, wy)
        for k, o in zip(leds, fields):
            if opt.fidelity == 0:
                W = o * w
            elif opt.fidelity == 1:
                W = o / (2.0 * np.maximum(np.sqrt(s), opt.eta_h)) * w
            else:
                W = scaling_map_slope(np.sqrt(s), opt) * o * w
            G = np.fft.fftshift(np.fft.fft2(W)) / (u * u * n * n)
            if want_tiles:
                tiles[k] = G
            g_psi += crop_adjoint(np.conj(p_eff) * G, geo, k)
            g_p += np.conj(crop(psi, geo, k)) * G
    g_p = g_p * mask
    return cost, g_psi, g_p, tiles


# ----------------------------------------------------------------------------
# Hessian regulariser (Eqs. 6-7) and its gradients (Eqs. 13-14)
# ----------------------------------------------------------------------------
def object_from_spectrum(psi):
    """O = IDFT_N(ifftshift(Psi)) (A1; Algorithm 1's O <- F_A^-1 Psi)."""
    return np.fft.ifft2(np.fft.ifftshift(psi))


def spectrum_from_object(obj):
    """Psi = fftshift(DFT_N(O)) (A1; Sec. 3.1)."""
    return np.fft.fftshift(np.fft.fft2(obj))


def hessian_cost_grad(psi, alpha, beta, opt: Options):
    """alpha L_A + beta L_Phi and its gradient with respect to conj(Psi).

      O = object_from_spectrum(Psi);  a = |O|;  phi = atan2(Im O, Re O)   (A12)
      (L_A, omega_a)   = huber(H a)                                     (Eq. 6)
      (L_Phi, omega_p) = huber(H phi)                                   (Eq. 7)
      q = alpha O/(2 max(a, eta_H)) H^T omega_a
        + beta (i/2) O/(a^2 + eta_H) H^T omega_p                        (Eqs. 13-14, A13)
      g_H = (1/A) fftshift(DFT_N(q))                                    (F_A^H)
    Returns (L_A, L_Phi, g_H).  L_A and L_Phi are not weighted by alpha/beta.
    """
    N = psi.shape[0]
    obj = object_from_spectrum(psi)
    a = np.abs(obj)
    ph = np.arctan2(obj.imag, obj.real)
    interior = np.zeros((N, N), dtype=bool)
    interior[1:-1, 1:-1] = True
    ha = hessian_op(a)
    cost_a, wa = huber(list(ha), opt.tau_h, opt.omega_iso)
    hp = hessian_op(ph)
    cost_p, wp = huber(list(hp), opt.tau_h, opt.omega_iso)
    L_A = float(np.sum(cost_a[interior]))
    L_P = float(np.sum(cost_p[interior]))
    wa = [w * interior for w in wa]
    wp = [w * interior for w in wp]
    ta = hessian_adj(*wa)
    tp = hessian_adj(*wp)
    q = alpha * obj / (2.0 * np.maximum(a, opt.eta_h)) * ta
    q = q + beta * 0.5j * obj / (a * a + opt.eta_h) * tp
    g = np.fft.fftshift(np.fft.fft2(q)) / (N * N)
    return L_A, L_P, g


# ----------------------------------------------------------------------------
# modified AdaBelief (Eq. 19)
# ----------------------------------------------------------------------------
def adabelief(x, g, mu, v, delta, t, opt: Options):
    """One step of Eq. 19 at iteration index t >= 1 (g is dL/d(conj x), A11).

      mu    = g1 mu + (1 - g1) g
      v     = g2 v + (1 - g2) |mu - g|^2
      mu^   = mu / (1 - g1^t);  v^ = v / (1 - g2^t)
      Delta = (sqrt(delta) + eta)/(sqrt(v^) + eta) * (g1 mu^ + (1 - g1) g)
      x     = x - Delta
      delta = g1 delta + (1 - g1) |Delta|^2
    Returns (x, mu, v, delta, Delta).
    """
    g1, g2, eta = opt.gamma1, opt.gamma2, opt.eta_opt
    mu = g1 * mu + (1.0 - g1) * g
    v = g2 * v + (1.0 - g2) * np.abs(mu - g) ** 2
    mu_hat = mu / (1.0 - g1 ** t)
    v_hat = v / (1.0 - g2 ** t)
    step = (np.sqrt(delta) + eta) / (np.sqrt(v_hat) + eta) * (g1 * mu_hat + (1.0 - g1) * g)
    x = x - step
    delta = g1 * delta + (1.0 - g1) * np.abs(step) ** 2
    return x, mu, v, delta, step


# ----------------------------------------------------------------------------
# pupil smoothing (note under Algorithm 1)
# ----------------------------------------------------------------------------
def gauss3():
    """3 x 3 Gaussian kernel of width (sigma) 1 pixel, normalised to sum 1."""
    g = np.exp(-0.5 * np.arange(-1, 2, dtype=np.float64) ** 2)
    k = np.outer(g, g)
    return k / k.sum()


def filter3(p):
    """G3 (x) P with zero padding outside the n x n grid."""
    k = gauss3()
    n0, n1 = p.shape
    pad = np.zeros((n0 + 2, n1 + 2), dtype=p.dtype)
    pad[1:-1, 1:-1] = p
    out = np.zeros_like(p)
    for dy in range(3):
        for dx in range(3):
            out += k[dy, dx] * pad[dy:dy + n0, dx:dx + n1]
    return out


# ----------------------------------------------------------------------------
# automatic regularisation weight (Eqs. 16-17, A10)
# ----------------------------------------------------------------------------
LAPLACE_KERNEL = np.array([[-1.0, 2.0, -1.0], [-2.0, 4.0, -2.0], [-1.0, 2.0, -1.0]])


def alpha_estimate(I, amplitude=False, opt: Options | None = None):
    """alpha = beta = (1/5) sqrt(pi/2) * mean_n mean_interior |I_n (x) L| (Eq. 16),
    or of sqrt(I_n) for the amplitude fidelity (Eq. 17), or of g(max(I_n, 0)) for
    the power and log maps of Sec. 6.3 (A17, when opt.fidelity is 2 or 3).
    'valid' 3x3 window."""
    I = np.asarray(I, dtype=np.float64)
    if opt is not None and opt.fidelity in (2, 3):
        I = scaling_map(np.maximum(I, 0.0), opt)
    elif amplitude or (opt is not None and opt.fidelity == 1):
        I = np.sqrt(np.maximum(I, 0.0))
    K, h, w = I.shape
    acc = np.zeros((K, h - 2, w - 2))
    for dy in range(3):
        for dx in range(3):
            acc += LAPLACE_KERNEL[dy, dx] * I[:, dy:dy + h - 2, dx:dx + w - 2]
    return 0.2 * math.sqrt(math.pi / 2.0) * float(np.mean(np.abs(acc)))


# ----------------------------------------------------------------------------
# state, initialisation (A9) and the iteration (Algorithm 1)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class State:
    psi: np.ndarray
    mu_psi: np.ndarray
    v_psi: np.ndarray
    delta_psi: np.ndarray
    pupil: np.ndarray
    mu_p: np.ndarray
    v_p: np.ndarray
    delta_p: np.ndarray
    t: int
    alpha: float
    beta: float

    def copy(self) -> "State":
        return State(**{f.name: (getattr(self, f.name).copy()
                                 if isinstance(getattr(self, f.name), np.ndarray)
                                 else getattr(self, f.name))
                        for f in dataclasses.fields(self)})


def centre_led(k_xy):
    """Index of the LED closest to the optical axis (lowest index on ties)."""
    k = np.asarray(k_xy, dtype=np.float64).reshape(-1, 2)
    return int(np.argmin(k[:, 0] ** 2 + k[:, 1] ** 2))


def init_state(I, geo: Geometry, k_xy, opt: Options) -> State:
    """Initial state (A9): Psi0 from the centre-LED image, P0 = 1 on S.

    Psi0 = u^2 * (fftshift(DFT_n(sqrt(max(I_c, 0)))) with its Nyquist row and
    column zeroed), placed at the centre LED's crop window; mu = v = 0;
    delta = s0^2; alpha, beta from Eq. 16/17 when negative in the options.
    """
    n, u, N = geo.n, geo.u, geo.N
    c = centre_led(k_xy)
    small = np.fft.fftshift(np.fft.fft2(np.sqrt(np.maximum(I[c // geo.mux], 0.0)))) * (u * u)
    small[0, :] = 0.0
    small[:, 0] = 0.0
    psi = crop_adjoint(small, geo, c)
    pupil = geo.support.astype(np.complex128)
    a_auto = None
    if opt.alpha < 0 or opt.beta < 0:
        a_auto = alpha_estimate(I, opt=opt)
    alpha = a_auto if opt.alpha < 0 else float(opt.alpha)
    beta = a_auto if opt.beta < 0 else float(opt.beta)
    return State(
        psi=psi,
        mu_psi=np.zeros((N, N), dtype=np.complex128),
        v_psi=np.zeros((N, N)),
        delta_psi=np.full((N, N), opt.s0_psi ** 2),
        pupil=pupil,
        mu_p=np.zeros((n, n), dtype=np.complex128),
        v_p=np.zeros((n, n)),
        delta_p=np.full((n, n), opt.s0_pupil ** 2),
        t=0, alpha=float(alpha), beta=float(beta))


def update_norms(g_psi, step):
    """(||g||, ||Delta Psi||) of one Psi update: the Euclidean norms over the N x N spectrum of
    the gradient used by Eq. 19 and of Psi^(t+1) - Psi^t = -Delta."""
    return float(np.sqrt(np.sum(np.abs(g_psi) ** 2))), float(np.sqrt(np.sum(np.abs(step) ** 2)))


def iteration(state: State, I, geo: Geometry, opt: Options, want=False, fidelity=None, norms=None):
    """One outer iteration of Algorithm 1 from state t to t+1.

    Gradients are evaluated at (Psi^t, P^t) (Sec. 3.3-3.4), then Psi and P are
    updated with Eq. 19; P is Gaussian-filtered before its update (A15).
    ``fidelity``, if given, replaces the call of fidelity_cost_grad (same
    arguments and results); oracle/parallel.py passes one that splits the LED
    sum over processes.  It is started before the Hessian branch is evaluated.
    ``norms``, if a list, gets the iteration's update_norms appended.
    Returns (new_state, costs=(L_fid, L_A, L_Phi) at state t, extras or None).
    """
    if fidelity is None:
        L_fid, g_fid, g_p, tiles = fidelity_cost_grad(state.psi, state.pupil, I, geo, opt,
                                                      want_tiles=want)
        L_A, L_P, g_h = hessian_cost_grad(state.psi, state.alpha, state.beta, opt)
    else:
        pending = fidelity(state.psi, state.pupil, I, geo, opt, want_tiles=want)
        L_A, L_P, g_h = hessian_cost_grad(state.psi, state.alpha, state.beta, opt)
        L_fid, g_fid, g_p, tiles = pending() if callable(pending) else pending
    g_psi = g_fid + g_h
    t = state.t + 1
    s = state.copy()
    s.t = t
    s.psi, s.mu_psi, s.v_psi, s.delta_psi, step = adabelief(
        state.psi, g_psi, state.mu_psi, state.v_psi, state.delta_psi, t, opt)
    if norms is not None:
        norms.append(update_norms(g_psi, step))
    if opt.learn_pupil:
        p_base = filter3(state.pupil) if opt.pupil_filter else state.pupil
        p_new, s.mu_p, s.v_p, s.delta_p, _ = adabelief(
            p_base, g_p, state.mu_p, state.v_p, state.delta_p, t, opt)
        s.pupil = p_new * geo.support
    extras = None
    if want:
        extras = dict(g_fid=g_fid, g_h=g_h, g_p=g_p, tiles=tiles)
    return s, (L_fid, L_A, L_P), extras


def run(state: State, I, geo: Geometry, opt: Options, n_iter: int, fidelity=None, norms=None):
    """n_iter iterations; returns (final state, costs [n_iter, 3]); ``norms``, if a list, gets each
    iteration's update_norms."""
    costs = []
    for _ in range(n_iter):
        state, c, _ = iteration(state, I, geo, opt, fidelity=fidelity, norms=norms)
        costs.append(c)
    return state, np.asarray(costs, dtype=np.float64).reshape(-1, 3)


def total_cost(costs, alpha, beta):
    """Eq. 8: L = L_fid + alpha L_A + beta L_Phi."""
    c = np.asarray(costs, dtype=np.float64)
    return c[..., 0] + alpha * c[..., 1] + beta * c[..., 2]


# ----------------------------------------------------------------------------
# evaluation of Sec. 4.1: degradations (Eqs. 2, 20), NL (Eq. 21), LSNR (Eq. 22)
# ----------------------------------------------------------------------------
def gaussian_kernel_periodic(n, waist_px):
    """G of Eq. 20 on an n x n periodic grid: exp(-2 r^2 / w^2) (w the 1/e^2 half-waist,
    A19), r the wrapped distance to pixel (0, 0), normalised to unit sum."""
    d = np.minimum(np.arange(n), n - np.arange(n)).astype(np.float64)
    r2 = d[None, :] ** 2 + d[:, None] ** 2
    g = np.exp(-2.0 * r2 / float(waist_px) ** 2)
    return g / g.sum()


def circular_convolve(f, g):
    """(g (x) f)[y, x] = sum_{a, b} g[a, b] f[(y - a) mod n, (x - b) mod n], summed directly."""
    n = f.shape[0]
    out = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            if g[a, b] != 0.0:
                out += g[a, b] * np.roll(np.roll(f, a, axis=0), b, axis=1)
    return out


def illumination_pattern(zeta, c, waist_px):
    """Uneven illumination of Eq. 20 for one image: (1 - c) + c * N(G (x) zeta), with N the
    min-max normalisation to [0, 1] (A19; N = 0 for a flat field) and (x) the circular
    convolution (A20)."""
    blur = circular_convolve(np.asarray(zeta, dtype=np.float64), gaussian_kernel_periodic(zeta.shape[0], waist_px))
    lo, hi = blur.min(), blur.max()
    norm = (blur - lo) / (hi - lo) if hi > lo else np.zeros_like(blur)
    return (1.0 - c) + c * norm


def degrade(I_clean, c=0.0, waist_px=15.0, zeta=None, background=None, gauss_a=0.0, xi=None,
            snp_density=0.0, u_snp=None):
    """Eqs. 2 and 20 with the random fields given: per image j,
      I_j = Lambda_j o I_clean_j + Omega_j + a xi_j,  Lambda_j = illumination_pattern(zeta_j)
    (Lambda = 1 when c = 0, Omega = 0 when background is None), then salt & pepper with the
    uniform field u: u < d/2 -> 0, d/2 <= u < d -> 1 (the 'salt & pepper' rule of the
    imnoise call of Sec. 4.1).  Arrays [K/M, n, n]; background [K/M]."""
    I = np.array(I_clean, dtype=np.float64, copy=True)
    for j in range(I.shape[0]):
        if c != 0.0:
            I[j] *= illumination_pattern(zeta[j], c, waist_px)
        if background is not None:
            I[j] += float(background[j])
        if gauss_a != 0.0:
            I[j] += gauss_a * np.asarray(xi[j], dtype=np.float64)
    if snp_density != 0.0:
        u = np.asarray(u_snp, dtype=np.float64)
        I = np.where(u < snp_density / 2.0, 0.0, np.where(u < snp_density, 1.0, I))
    return I


def darkfield_images(geo: Geometry, na, wavelength_um):
    """Dark-field images of Eq. 21: image j when every LED lighting it has its illumination
    frequency outside the pupil, |c_n| dk > NA / lambda."""
    r = np.sqrt(np.sum(geo.offsets.astype(np.float64) ** 2, axis=1)) * geo.dk
    dark_led = r > float(na) / float(wavelength_um)
    return dark_led.reshape(geo.n_images, geo.mux).all(axis=1)


def noise_level(I_simu, I_noised, dark):
    """NL of Eq. 21 in percent: mean over the dark-field images of
    ||I_simu - I_noised||_1 / ||I_simu||_1."""
    I_simu = np.asarray(I_simu, dtype=np.float64)
    I_noised = np.asarray(I_noised, dtype=np.float64)
    idx = np.flatnonzero(np.asarray(dark))
    if idx.size == 0:
        return 0.0
    ratios = [np.sum(np.abs(I_simu[j] - I_noised[j])) / np.sum(np.abs(I_simu[j])) for j in idx]
    return 100.0 * float(np.mean(ratios))


def lsnr(rec, truth):
    """LSNR of Eq. 22 in dB: max over b of 10 log10(||truth||^2 / ||truth - (rec + b)||^2);
    the maximising b is the mean of truth - rec (least squares in one constant)."""
    t = np.asarray(truth, dtype=np.float64).ravel()
    d = t - np.asarray(rec, dtype=np.float64).ravel()
    b = d.mean()
    return 10.0 * math.log10(float(np.sum(t * t)) / float(np.sum((d - b) ** 2)))


def object_quality(obj_rec, obj_true):
    """(LSNR of the amplitude, LSNR of the phase) of a reconstruction against the truth, after
    removing the unobservable global phase: obj_rec is multiplied by e^{i phi0} with
    phi0 = arg sum conj(obj_rec) obj_true (the least-squares global phase)."""
    obj_rec = np.asarray(obj_rec, dtype=np.complex128)
    obj_true = np.asarray(obj_true, dtype=np.complex128)
    phi0 = np.angle(np.sum(np.conj(obj_rec) * obj_true))
    aligned = obj_rec * np.exp(1j * phi0)
    return lsnr(np.abs(aligned), np.abs(obj_true)), lsnr(np.angle(aligned), np.angle(obj_true))
