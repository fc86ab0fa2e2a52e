"""Writes fp32_spread_<case>.json: how far the FP64 oracle's own run of a workload
(Algorithm 1) moves when noise of the size of the GPU path's rounding is injected.

The FP32 model injects noise at the two places where rounding enters an FP32
implementation: every element of the stored state Psi and P is multiplied by
(1 + 1e-7 xi) after the start state and after every iteration, and the object
O = F_A^-1 Psi of the Hessian branch gets 1e-7 rms(|O|) zeta added per element each time it
is formed (xi, zeta complex standard normal; an FP32 FFT of N^2 points rounds to about
2^-24 sqrt(log2 N^2) = 2.4e-7 of the rms value at N = 256).  The tensor-core model adds,
on top, 2e-5 rms(|o_n|) zeta to every LED field o_n of Eq. 1: a BF16 hi + lo product keeps
about 16 significant bits (2^-16 = 1.5e-5), once for the inverse and once for the forward
tile transform.

The spread (relative L2 distance of the perturbed runs from the unperturbed one, and the
largest relative difference of the per-iteration costs) bounds how closely any
implementation with that rounding can follow the FP64 trajectory.  Calls only the oracle
and the seeded input generator.  Run from the repository root:
    python tests/golden/make_fp32_spread.py w0      # 20 iterations from the initial state
    python tests/golden/make_fp32_spread.py w3      # 200 iterations from the t = 3 state
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
import oracle.elfpie_oracle as OE  # noqa: E402
from _cases import case, oracle_state_to_f32, rel  # noqa: E402

EPS = 1e-7
EPS_TC = 2e-5
KEYS = ("psi", "pupil", "L_fid", "L_A", "L_P")


def perturb(st, rng):
    s = st.copy()
    for k in ("psi", "pupil"):
        x = getattr(s, k)
        xi = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        setattr(s, k, x * (1.0 + EPS * xi))
    return s


def additive_noise(orig, rng, eps):
    def f(*a):
        o = orig(*a)
        r = np.sqrt(np.mean(np.abs(o) ** 2))
        return o + eps * r * (rng.standard_normal(o.shape) + 1j * rng.standard_normal(o.shape))
    return f


def run(st0, I, geo, opt, checkpoints, rng=None, model="fp32"):
    """Iterations from st0; the state and costs at each checkpoint (iteration counts)."""
    saved = (OE.object_from_spectrum, OE.forward_field)
    out = {}
    costs = []
    try:
        st = st0
        if rng is not None:
            st = perturb(st, rng)
            OE.object_from_spectrum = additive_noise(saved[0], rng, EPS)
            if model == "tc":
                OE.forward_field = additive_noise(saved[1], rng, EPS_TC)
        for it in range(1, checkpoints[-1] + 1):
            st, cc, _ = O.iteration(st, I, geo, opt)
            costs.append(cc)
            if rng is not None:
                st = perturb(st, rng)
            if it in checkpoints:
                out[it] = (st, np.asarray(costs))
    finally:
        OE.object_from_spectrum, OE.forward_field = saved
    return out


def main():
    which = sys.argv[1] if len(sys.argv) > 1 else "w0"
    c = case(which)
    I = c["I"].astype(np.float64)
    opt = O.Options()
    st0 = O.init_state(I, c["geo"], c["k_xy"], opt)
    if which == "w0":
        start, checkpoints, models, seeds = "the initial state (t = 0)", [c["iters"]], ["fp32"], 8
    else:
        st0, _ = O.run(st0, I, c["geo"], opt, 3)
        st0 = oracle_state_to_f32(st0)
        start, checkpoints, models, seeds = "the oracle's t = 3 state rounded to FP32", [50, 100, 150, 200], \
            ["fp32", "tc"], 3
    ref = run(st0, I, c["geo"], opt, checkpoints)
    result = {}
    for model in models:
        per_it = {it: [] for it in checkpoints}
        for seed in range(seeds):
            got = run(st0, I, c["geo"], opt, checkpoints, np.random.default_rng([2209, seed]), model)
            for it in checkpoints:
                st, costs = got[it]
                st_r, costs_r = ref[it]
                ce = np.abs(costs - costs_r) / np.abs(costs_r)
                per_it[it].append(dict(seed=seed, psi=rel(st.psi, st_r.psi), pupil=rel(st.pupil, st_r.pupil),
                                       L_fid=float(ce[:, 0].max()), L_A=float(ce[:, 1].max()),
                                       L_P=float(ce[:, 2].max())))
                print(model, it, per_it[it][-1], flush=True)
        result[model] = {str(it): {"runs": r, "max": {k: max(x[k] for x in r) for k in KEYS},
                                   "median": {k: float(np.median([x[k] for x in r])) for k in KEYS}}
                         for it, r in per_it.items()}
    out = {
        "what": f"relative L2 distance of perturbed FP64 oracle runs from the unperturbed one, workload "
                f"{c['name']}, from {start}, at the listed iteration counts; per-iteration cost differences "
                f"are the largest relative difference up to that count",
        "models": {"fp32": f"state (Psi, P) times 1 + {EPS:g} xi after every iteration, {EPS:g} rms(|O|) "
                           "complex noise added to O in every Hessian evaluation",
                   "tc": f"fp32 plus {EPS_TC:g} rms(|o_n|) complex noise added to every LED field o_n"},
        "written_by": "tests/golden/make_fp32_spread.py (oracle and input generator only)",
        "seeds": seeds,
        "spread": result,
    }
    with open(os.path.join(HERE, f"fp32_spread_{which}.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
