"""Differentiation form: ElfCost (torch.autograd.Function over elf_cost_grad).

At the workload sizes of the differentiation check (64 x 64 images, 7 x 7 LEDs,
256 x 256 spectrum), on a developed state:
  * autograd gradients / 2 equal the FP64 oracle's dL/d(conj Psi), dL/d(conj P)
    (relative L2 2e-3, as the other gradient parity tests);
  * central finite differences of the GPU cost along 32 seeded complex
    directions (for Psi and for P) match 2 Re<g, d>: Richardson-extrapolated
    central differences with steps 2e-3 and 1e-3 of |Psi|; median 1e-3, 90th
    percentile 1e-2.  FP32 cannot resolve steps much below 1e-3 of
    |Psi|, and with the default smoothing radii the Huber-smoothed L1 terms
    curve on a scale of tau, so the FP64 oracle's own differences only converge
    at steps near 1e-6; this check therefore uses tau = 0.1 (any tau is a valid
    test of the gradient code), where the FP64 differences at these steps are
    within 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E
from paper_2209_14671_gb300 import inputs as IN

from _cases import case, load_state, oracle_state_to_f32, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OPTS = dict(tau_fid=1e-3, tau_h=1e-3)
OPTS_FD = dict(tau_fid=0.1, tau_h=0.1)


def _setup(opts):
    B.build()
    E.load()
    from paper_2209_14671_gb300.autograd import ElfCost
    c = case("w2")
    I = c["I"].astype(np.float64)
    opt = O.Options(**opts)
    st = O.init_state(I, c["geo"], c["k_xy"], opt)
    st, _ = O.run(st, I, c["geo"], opt, 3)
    st = oracle_state_to_f32(st)
    elf = E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], options=opts)
    elf.set_measurements(c["I"])
    load_state(elf, st)
    return c, st, opt, elf, ElfCost(elf)


@pytest.fixture(scope="module")
def setup():
    r = _setup(OPTS)
    yield r
    r[3].close()


@pytest.fixture(scope="module")
def setup_fd():
    r = _setup(OPTS_FD)
    yield r
    r[3].close()


def test_autograd_gradients_match_oracle(setup):
    c, st, opt, elf, cost = setup
    dev = torch.device("cuda:0")
    psi = torch.from_numpy(st.psi.astype(np.complex64)).to(dev).requires_grad_(True)
    pup = torch.from_numpy(st.pupil.astype(np.complex64)).to(dev).requires_grad_(True)
    L = cost(psi, pup)
    L.backward()
    I = c["I"].astype(np.float64)
    L_fid, g_fid, g_p, _ = O.fidelity_cost_grad(st.psi, st.pupil, I, c["geo"], opt)
    L_A, L_P, g_h = O.hessian_cost_grad(st.psi, st.alpha, st.beta, opt)
    L_ref = L_fid + st.alpha * L_A + st.beta * L_P
    e_L = abs(L.item() - L_ref) / L_ref
    e_psi = rel(psi.grad.cpu().numpy() / 2, g_fid + g_h)
    e_p = rel(pup.grad.cpu().numpy() / 2, g_p)
    print(f"autograd vs oracle: L {e_L:.2e} g_psi {e_psi:.2e} g_pupil {e_p:.2e}")
    assert e_L < 1e-5 and e_psi < 2e-3 and e_p < 2e-3


def test_autograd_matches_central_differences(setup_fd):
    c, st, opt, elf, cost = setup_fd
    dev = torch.device("cuda:0")
    psi0 = st.psi
    pup0 = st.pupil
    psi = torch.from_numpy(psi0.astype(np.complex64)).to(dev).requires_grad_(True)
    pup = torch.from_numpy(pup0.astype(np.complex64)).to(dev).requires_grad_(True)
    cost(psi, pup).backward()
    g_psi = psi.grad.cpu().numpy().astype(np.complex128) / 2
    g_pup = pup.grad.cpu().numpy().astype(np.complex128) / 2
    dirs = IN.complex_directions(psi0.shape, 32, 2)
    pdirs = IN.complex_directions(pup0.shape, 32, 2) * c["geo"].support

    def L(p, q):
        with torch.no_grad():
            return cost(torch.from_numpy(p.astype(np.complex64)).to(dev),
                        torch.from_numpy(q.astype(np.complex64)).to(dev)).item()
    def central(x0, d, h, is_psi):
        if is_psi:
            return (L(x0 + h * d, pup0) - L(x0 - h * d, pup0)) / (2 * h)
        return (L(psi0, x0 + h * d) - L(psi0, x0 - h * d)) / (2 * h)
    errs = []
    for k in range(32):
        for (x0, g, d, is_psi) in ((psi0, g_psi, dirs[k], True), (pup0, g_pup, pdirs[k], False)):
            d = d * (np.linalg.norm(x0) / np.linalg.norm(d))
            h = 2e-3
            # Richardson extrapolation of two central differences: O(h^4) truncation with a
            # step large enough that the FP32 cost's rounding noise stays far below the signal
            fd = (4.0 * central(x0, d, h / 2, is_psi) - central(x0, d, h, is_psi)) / 3.0
            an = 2.0 * np.real(np.vdot(g, d))
            errs.append(abs(fd - an) / abs(an))
    errs = np.array(errs)
    print(f"finite differences: median {np.median(errs):.2e} 90th percentile {np.percentile(errs, 90):.2e} "
          f"max {errs.max():.2e}")
    # a wrong gradient term gives O(1) errors in every direction; the few directions nearly
    # orthogonal to the gradient carry the FP32 rounding noise of the cost
    assert np.median(errs) < 1e-3 and np.percentile(errs, 90) < 1e-2 and errs.max() < 0.2
