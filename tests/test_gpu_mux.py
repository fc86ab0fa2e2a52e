"""Multiplexed illumination (Eq. 1 with M LEDs per measured image) on the CUDA path
against the FP64 oracle, through the C ABI.

Image j is lit by LEDs jM .. jM+M-1.  The measurements are the oracle's multiplexed
forward model of the workload objects plus seeded Gaussian noise (sigma 1e-3), so both
sides see the same float32 images.  Bounds are those of the sequential path: forward
model and costs 1e-5, gradients 2e-3, state after one iteration 1e-5 (relative L2).
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E

from _cases import case, load_state, oracle_state_to_f32, rel

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-5
TOL_GRAD = 2e-3
TOL_STATE = 1e-5

# (base case, M): 9 LEDs as 3 images of 3, 25 LEDs as 5 of 5, the 49-LED workload as 7 of 7,
# and the 225-LED / 256 x 256 workload as 45 images of 5
MUX_CASES = [("tiny16", 3), ("small32", 5), ("w0", 7), ("w1", 5)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    E.load()


@functools.lru_cache(maxsize=None)
def mux_case(name, M):
    c = dict(case(name))
    geo = O.make_geometry(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], mux=M)
    I = O.forward_intensity(O.spectrum_from_object(c["obj"]), geo.support.astype(complex), geo)
    g = np.random.default_rng([97, M, c["n"]])
    c["I"] = (I + 1e-3 * g.standard_normal(I.shape)).astype(np.float32)
    c["geo"] = geo
    c["M"] = M
    return c


_developed = {}


def developed(name, M, **opts):
    key = (name, M, tuple(sorted(opts.items())))
    if key not in _developed:
        c = mux_case(name, M)
        opt = O.Options(**opts)
        I = c["I"].astype(np.float64)
        st = O.init_state(I, c["geo"], c["k_xy"], opt)
        st, _ = O.run(st, I, c["geo"], opt, 3)
        _developed[key] = oracle_state_to_f32(st)
    return _developed[key]


def make_elf(c, **opts):
    return E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], options=opts or None, mux=c["M"])


@pytest.mark.parametrize("name,M", MUX_CASES)
def test_multiplexed_forward_model(name, M):
    c = mux_case(name, M)
    ref = O.forward_intensity(O.spectrum_from_object(c["obj"]), c["geo"].support.astype(complex), c["geo"])
    with make_elf(c) as elf:
        out = elf.simulate(c["obj"].astype(np.complex64))
    assert out.shape == (c["geo"].n_images, c["n"], c["n"])
    e = rel(out, ref)
    print(name, M, f"simulate {e:.2e}")
    assert e < TOL_FWD


@pytest.mark.parametrize("name,M", MUX_CASES)
def test_multiplexed_initial_state_and_alpha(name, M):
    c = mux_case(name, M)
    I = c["I"].astype(np.float64)
    st = O.init_state(I, c["geo"], c["k_xy"], O.Options())
    with make_elf(c) as elf:
        elf.set_measurements(c["I"])
        a_gpu, _ = elf.get_weights()
        psi = elf.get_spectrum()
    e = dict(alpha=abs(a_gpu - st.alpha) / st.alpha, psi=rel(psi, st.psi))
    print(name, M, " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["alpha"] < 1e-6 and e["psi"] < TOL_FWD


@pytest.mark.parametrize("name,M", MUX_CASES)
@pytest.mark.parametrize("variant", [dict(), dict(fidelity=1), dict(fidelity=3, omega_iso=0)])
def test_multiplexed_cost_and_gradients(name, M, variant):
    c = mux_case(name, M)
    st = developed(name, M, **variant)
    I = c["I"].astype(np.float64)
    opt = O.Options(**variant)
    L_fid, g_fid, g_p, tiles = O.fidelity_cost_grad(st.psi, st.pupil, I, c["geo"], opt, want_tiles=True)
    L_A, L_P, g_h = O.hessian_cost_grad(st.psi, st.alpha, st.beta, opt)
    with make_elf(c, **variant) as elf:
        elf.set_measurements(c["I"])
        load_state(elf, st)
        costs, g_psi, g_pup = elf.cost_grad(st.psi.astype(np.complex64), st.pupil.astype(np.complex64))
        G = elf.get_tile_grads()
        sup = elf.get_support()
    G_ref = tiles.reshape(tiles.shape[0], -1)[:, sup]
    e = dict(L_fid=abs(costs[0] - L_fid) / L_fid, L_A=abs(costs[1] - L_A) / L_A, G=rel(G, G_ref),
             g_psi=rel(g_psi, g_fid + g_h), g_p=rel(g_pup, g_p))
    print(name, M, variant, " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["L_fid"] < TOL_FWD and e["L_A"] < TOL_FWD
    assert e["G"] < TOL_GRAD and e["g_psi"] < TOL_GRAD and e["g_p"] < TOL_GRAD


@pytest.mark.parametrize("name,M", MUX_CASES)
def test_multiplexed_one_iteration(name, M):
    c = mux_case(name, M)
    st = developed(name, M)
    I = c["I"].astype(np.float64)
    ref, costs_ref, _ = O.iteration(st, I, c["geo"], O.Options())
    with make_elf(c) as elf:
        elf.set_measurements(c["I"])
        load_state(elf, st)
        elf.step(1)
        out = elf.get_state()
        costs = elf.get_costs()[-1]
    e = dict(psi=rel(out["psi"], ref.psi), pupil=rel(out["pupil"], ref.pupil),
             cost=float(np.max(np.abs(costs - np.asarray(costs_ref)) / np.asarray(costs_ref))))
    print(name, M, " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["psi"] < TOL_STATE and e["pupil"] < TOL_STATE and e["cost"] < TOL_FWD


def test_multiplexed_runs_are_bitwise_reproducible():
    c = mux_case("w0", 7)
    out = []
    for _ in range(2):
        with make_elf(c) as elf:
            elf.set_measurements(c["I"])
            elf.step(5)
            out.append(elf.get_spectrum())
    assert np.array_equal(out[0], out[1])


def test_multiplexed_geometry_is_validated():
    c = dict(case("small32"))  # 25 LEDs
    for M, opts in ((2, {}), (26, {})):
        with pytest.raises(E.ElfError) as ei:
            E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], mux=M, options=opts or None)
        assert ei.value.code == E.ELF_EINVAL
    w3 = case("w3")  # n = 128: the tensor-core form takes sequential images only
    with pytest.raises(E.ElfError) as ei:
        E.Elf(w3["n"], w3["u"], w3["k_xy"], w3["na"], w3["wl"], w3["dx"], mux=5, options=dict(tile_dft=1))
    assert ei.value.code == E.ELF_EINVAL
