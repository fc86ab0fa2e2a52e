"""LED sharding of the iteration on the GPU (elf_shard_* through the C ABI, shard.py).

Eqs. 9 and 18 sum per-LED terms (Sec. 3.4).  Handles of the same problem that each run
the tile work of one block of LEDs, exchange the per-LED results and finish the iteration
must end every iteration in exactly the state of one handle's elf_step: the per-LED
results travel unsummed and every sum over LEDs runs after the exchange in LED order.
Checked bitwise for 2, 3 and 4 blocks (even, uneven, one empty), from a developed oracle
state, against elf_step and against the FP64 oracle; then with two processes on the one
GPU exchanging through a gloo process group.
"""
import datetime
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E
from paper_2209_14671_gb300 import shard as SH

from _cases import case, load_state, oracle_state_to_f32, rel

pytestmark = pytest.mark.gpu

ITERS = 3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    E.load()


def _developed(name, iters=3):
    c = case(name)
    I = c["I"].astype(np.float64)
    opt = O.Options()
    st = O.init_state(I, c["geo"], c["k_xy"], opt)
    st, _ = O.run(st, I, c["geo"], opt, iters)
    return c, oracle_state_to_f32(st)


def _make(c, st, **kw):
    elf = E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], **kw)
    elf.set_measurements(c["I"])
    load_state(elf, st)
    return elf


def _snapshot(elf):
    s = elf.get_state()
    return {k: np.asarray(v).copy() for k, v in s.items() if isinstance(v, np.ndarray)}, elf.get_costs()


def _sharded_in_one_process(c, st, world, iters):
    """`world` handles as ranks in one process; the exchange is device-to-device through torch buffers."""
    import torch
    elfs = [_make(c, st) for _ in range(world)]
    blocks = SH.led_blocks(elfs[0].K, world)
    row = elfs[0].shard_row_floats()
    for _ in range(iters):
        bufs = []
        for e, (k0, k1) in zip(elfs, blocks):
            e.shard_tiles(k0, k1)
            buf = torch.empty(max(1, (k1 - k0) * row), dtype=torch.float32, device="cuda")
            if k1 > k0:
                e.shard_export(k0, k1, buf)
            bufs.append(buf)
        torch.cuda.synchronize()
        for r, e in enumerate(elfs):
            for q, (k0, k1) in enumerate(blocks):
                if q != r and k1 > k0:
                    e.shard_import(k0, k1, bufs[q])
            e.shard_finish()
    out = [_snapshot(e) for e in elfs]
    for e in elfs:
        e.close()
    return out


@pytest.mark.parametrize("name,world", [("w0", 2), ("w0", 3), ("small32", 4), ("single_led", 2), ("w1", 4)])
def test_sharded_iterations_equal_elf_step_bitwise(name, world):
    c, st = _developed(name)
    with _make(c, st) as ref:
        ref.step(ITERS)
        want, costs_want = _snapshot(ref)
    for r, (got, costs) in enumerate(_sharded_in_one_process(c, st, world, ITERS)):
        for k in want:
            assert np.array_equal(got[k], want[k]), (name, world, r, k)
        assert np.array_equal(costs, costs_want), (name, world, r)


def test_sharded_iteration_matches_oracle():
    c, st = _developed("w0")
    I = c["I"].astype(np.float64)
    ref, costs_ref, _ = O.iteration(st, I, c["geo"], O.Options())
    (got, costs), _ = _sharded_in_one_process(c, st, 2, 1)
    e = dict(psi=rel(got["psi"], ref.psi), pupil=rel(got["pupil"], ref.pupil),
             cost=float(np.max(np.abs(costs[-1] - np.asarray(costs_ref)) / np.asarray(costs_ref))))
    print("sharded one iteration vs oracle", e)
    assert e["psi"] < 1e-5 and e["pupil"] < 1e-5 and e["cost"] < 1e-5


def test_shard_call_order_and_arguments():
    c, st = _developed("small32", 2)
    with _make(c, st) as elf:
        with pytest.raises(E.ElfError) as ei:
            elf.shard_finish()
        assert ei.value.code == E.ELF_ESTATE
        with pytest.raises(E.ElfError) as ei:
            elf.shard_tiles(0, elf.K + 1)
        assert ei.value.code == E.ELF_EINVAL
        elf.shard_tiles(0, elf.K)
        for call in (lambda: elf.step(1), lambda: elf.shard_tiles(0, 1)):
            with pytest.raises(E.ElfError) as ei:
                call()
            assert ei.value.code == E.ELF_ESTATE
        elf.shard_finish()
        elf.step(1)
    with E.Elf(c["n"], c["u"], c["k_xy"][:24], c["na"], c["wl"], c["dx"], mux=2) as mx:
        with pytest.raises(E.ElfError) as ei:
            mx.shard_tiles(0, 2)
        assert ei.value.code == E.ELF_EINVAL


# ------------------------------------------------------------ two processes, gloo, one GPU
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, state_path, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        E.load()
        c = case(name)
        z = np.load(state_path)
        st = O.State(psi=z["psi"], mu_psi=z["mu_psi"], v_psi=z["v_psi"], delta_psi=z["delta_psi"], pupil=z["pupil"],
                     mu_p=z["mu_p"], v_p=z["v_p"], delta_p=z["delta_p"], t=int(z["t"]), alpha=float(z["alpha"]),
                     beta=float(z["beta"]))
        torch.cuda.set_device(0)
        elf = _make(c, st, stream=torch.cuda.current_stream())
        sh = SH.ShardedElf(elf, rank=rank, world=world)
        sh.step(ITERS)
        got, costs = _snapshot(elf)
        np.savez(out_path, costs=costs, exchanged=sh.exchanged_bytes, **got)
        elf.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_with_gloo_equal_elf_step(tmp_path):
    import torch.multiprocessing as mp
    c, st = _developed("w0")
    state_path = str(tmp_path / "state.npz")
    np.savez(state_path, psi=st.psi, mu_psi=st.mu_psi, v_psi=st.v_psi, delta_psi=st.delta_psi, pupil=st.pupil,
             mu_p=st.mu_p, v_p=st.v_p, delta_p=st.delta_p, t=st.t, alpha=st.alpha, beta=st.beta)
    with _make(c, st) as ref:
        ref.step(ITERS)
        want, costs_want = _snapshot(ref)
        S, K = ref.S, ref.K
    port = _free_port()
    ctx = mp.get_context("spawn")
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(2)]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, "w0", state_path, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(2):
        z = np.load(outs[r])
        for k in want:
            assert np.array_equal(z[k], want[k]), (r, k)
        assert np.array_equal(z["costs"], costs_want), r
        # 3 iterations x 2 ranks x the longer block (25 of 49 LEDs) x (S + cluster) complex values
        assert int(z["exchanged"]) == ITERS * 2 * 25 * (S + 2) * 8
