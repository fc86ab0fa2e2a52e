"""Precision form: the tile transforms as tensor-core GEMMs (tcgen05, BF16 3-term
split, FP32 accumulation; elf_options.tile_dft = 1) on the 128 x 128 / 225-LED
workload, against the FP64 oracle and against the FP32 FFT path.

The BF16 hi + lo pair carries 16 significant bits, so each product is exact to
about 2^-16 relative; sums over 64-128 terms keep the tile transforms within
~1e-5 relative.  Bounds (relative L2): forward-model tile gradients 1e-3, cost
1e-4, state after one iteration from a developed state 1e-5 (the update
contracts gradient errors by |Delta Psi| / |Psi|).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E

from _cases import case, load_state, oracle_state_to_f32, rel

pytestmark = pytest.mark.gpu


def _spread(model, at):
    """The FP64 oracle's own spread on this workload under the given noise model (largest of the
    seeded perturbed runs), written by tests/golden/make_fp32_spread.py."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp32_spread_w3.json")
    return json.load(open(path))["spread"][model][str(at)]["max"]


@pytest.fixture(scope="module")
def w3():
    B.build()
    E.load()
    c = case("w3")
    I = c["I"].astype(np.float64)
    opt = O.Options()
    st = O.init_state(I, c["geo"], c["k_xy"], opt)
    st, _ = O.run(st, I, c["geo"], opt, 3)
    return c, oracle_state_to_f32(st), opt


def _elf(c, tile_dft, **kw):
    return E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], options=dict(tile_dft=tile_dft, **kw))


def test_tensor_core_gradients_match_oracle(w3):
    c, st, opt = w3
    I = c["I"].astype(np.float64)
    L_fid, g_fid, g_p, tiles = O.fidelity_cost_grad(st.psi, st.pupil, I, c["geo"], opt, want_tiles=True)
    L_A, L_P, g_h = O.hessian_cost_grad(st.psi, st.alpha, st.beta, opt)
    out = {}
    for td in (0, 1):
        with _elf(c, td) as elf:
            elf.set_measurements(c["I"])
            load_state(elf, st)
            costs, g_psi, g_pup = elf.cost_grad(st.psi.astype(np.complex64), st.pupil.astype(np.complex64))
            G = elf.get_tile_grads()
            sup = elf.get_support()
        G_ref = tiles.reshape(tiles.shape[0], -1)[:, sup]
        out[td] = dict(L_fid=abs(costs[0] - L_fid) / L_fid, G=rel(G, G_ref), g_psi=rel(g_psi, g_fid + g_h),
                       g_p=rel(g_pup, g_p))
        print(f"tile_dft={td}: " + " ".join(f"{k} {v:.2e}" for k, v in out[td].items()))
    e = out[1]
    assert e["L_fid"] < 1e-4 and e["G"] < 1e-3 and e["g_psi"] < 2e-3 and e["g_p"] < 2e-3


def test_tensor_core_iteration_matches_oracle(w3):
    c, st, opt = w3
    I = c["I"].astype(np.float64)
    ref, costs_ref, _ = O.iteration(st, I, c["geo"], opt)
    with _elf(c, 1) as elf:
        elf.set_measurements(c["I"])
        load_state(elf, st)
        elf.step(1)
        s = elf.get_state()
        costs = elf.get_costs()[-1]
    e = dict(psi=rel(s["psi"], ref.psi), pupil=rel(s["pupil"], ref.pupil),
             cost=float(np.max(np.abs(costs - np.asarray(costs_ref)) / np.asarray(costs_ref))))
    print("tile_dft=1 one iteration: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["psi"] < 1e-5 and e["pupil"] < 1e-5 and e["cost"] < 1e-4


def test_tensor_core_path_rejects_unsupported_sizes():
    c = case("w0")  # n = 64
    with pytest.raises(E.ElfError) as ei:
        _elf(c, 1)
    assert ei.value.code == E.ELF_EINVAL


def test_full_run_against_oracle(w3):
    """The workload's full run (200 iterations, after the 3 of the developed state) on both tile
    paths; relative L2 of Psi and P against the FP64 oracle, reported every 50 iterations.

    The iteration amplifies small state differences, so a run drifts from FP64 by more than its
    per-iteration error.  The FP64 oracle itself, with noise of the FP32 path's rounding size
    injected into its state and its object, ends 200 iterations at a spread of Psi 1.2e-4 and
    P 4.9e-4 from the noiseless run; with the tensor-core model's noise (2e-5 of every LED field
    as well) at Psi 2.9e-4 and P 1.1e-2 (tests/golden/fp32_spread_w3.json).  Bounds on the final
    state: FFT path Psi 1e-4 (the full-run bound of the contract, which this run meets) and P twice
    the FP32 spread; tensor-core path Psi twice its spread and P 3e-3, tighter than twice its spread,
    as a guard on the measured 1.6e-3."""
    c, st, opt = w3
    I = c["I"].astype(np.float64)
    refs = {}
    ref = st
    for it in (50, 100, 150, 200):
        ref, _ = O.run(ref, I, c["geo"], opt, 50)
        refs[it] = ref
    errs = {}
    for td in (0, 1):
        with _elf(c, td) as elf:
            elf.set_measurements(c["I"])
            load_state(elf, st)
            for it in (50, 100, 150, 200):
                elf.step(50)
                s = elf.get_state()
                errs[(td, it)] = (rel(s["psi"], refs[it].psi), rel(s["pupil"], refs[it].pupil))
                print(f"tile_dft={td} after {it} iterations: psi {errs[(td, it)][0]:.2e} "
                      f"pupil {errs[(td, it)][1]:.2e}")
    sp32 = _spread("fp32", 200)
    sptc = _spread("tc", 200)
    assert errs[(0, 200)][0] < 1e-4 and errs[(0, 200)][1] < 2.0 * sp32["pupil"]
    assert errs[(1, 200)][0] < 2.0 * sptc["psi"] and errs[(1, 200)][1] < 3e-3


@pytest.mark.parametrize("variant", [dict(fidelity=2, g_exponent=0.375), dict(fidelity=3)])
def test_tensor_core_scaling_maps_match_oracle(w3, variant):
    """The Sec. 6.3 power and log fidelities on the tensor-core tile path: one iteration from the
    oracle state developed under the same fidelity, against the FP64 oracle."""
    c, _, _ = w3
    I = c["I"].astype(np.float64)
    opt = O.Options(**variant)
    st = O.init_state(I, c["geo"], c["k_xy"], opt)
    st, _ = O.run(st, I, c["geo"], opt, 3)
    st = oracle_state_to_f32(st)
    ref, costs_ref, _ = O.iteration(st, I, c["geo"], opt)
    with _elf(c, 1, **variant) as elf:
        elf.set_measurements(c["I"])
        load_state(elf, st)
        elf.step(1)
        s = elf.get_state()
        costs = elf.get_costs()[-1]
    e = dict(psi=rel(s["psi"], ref.psi), pupil=rel(s["pupil"], ref.pupil),
             cost=float(np.max(np.abs(costs - np.asarray(costs_ref)) / np.asarray(costs_ref))))
    print(variant, "tile_dft=1 one iteration: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["psi"] < 1e-5 and e["pupil"] < 1e-5 and e["cost"] < 1e-4
