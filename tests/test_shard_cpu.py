"""LED sharding, host side (paper_2209_14671_gb300/shard.py), with world-size 2 and 3 gloo
process groups on the CPU.

A fake handle stands in for the library: its "tile results" of LED k are a function of k
and of the state, and its "finish" folds all K results into the state in LED order.  The
sharded run on several ranks must leave every rank with exactly the state of one process
running all LEDs, for even and uneven partitions and for ranks with no LEDs; a rank that
dies before the exchange must make the others fail instead of hang.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2209_14671_gb300 import shard as SH


class FakeHandle:
    """Tile results of LED k: row k of a deterministic function of (k, state); finish adds them
    to the state in LED order (a non-associative float32 sum, so any other order would show)."""

    def __init__(self, K, S=5, C=2):
        self.K, self.S, self.C = K, S, C
        self.state = np.linspace(0.5, 1.5, S).astype(np.float32)
        self.rows = np.zeros((K, 2 * (S + C)), np.float32)
        self.open = False

    def shard_row_floats(self):
        return 2 * (self.S + self.C)

    def _row(self, k):
        g = np.random.default_rng(k).standard_normal(2 * (self.S + self.C)).astype(np.float32)
        return (g * (1.0 + self.state.mean()) * 1e3 ** (k % 3)).astype(np.float32)

    def shard_tiles(self, k0, k1):
        assert not self.open
        for k in range(k0, k1):
            self.rows[k] = self._row(k)
        self.open = True

    def _block(self, k0, k1):
        G = self.rows[k0:k1, :2 * self.S].reshape(-1)
        C = self.rows[k0:k1, 2 * self.S:].reshape(-1)
        return np.concatenate([G, C])  # the library's export layout: G of all LEDs, then the cost pairs

    def shard_export(self, k0, k1, out):
        out.copy_(torch.from_numpy(self._block(k0, k1)))
        return out

    def shard_import(self, k0, k1, src):
        x = src.numpy()
        n = k1 - k0
        G = x[:n * 2 * self.S].reshape(n, 2 * self.S)
        C = x[n * 2 * self.S:].reshape(n, 2 * self.C)
        self.rows[k0:k1, :2 * self.S] = G
        self.rows[k0:k1, 2 * self.S:] = C

    def shard_finish(self):
        assert self.open
        acc = np.zeros(2 * (self.S + self.C), np.float32)
        for k in range(self.K):
            acc = acc + self.rows[k]
        self.state = (self.state + 1e-3 * acc[:self.S]).astype(np.float32)
        self.open = False

    def step(self, n):
        for _ in range(n):
            self.shard_tiles(0, self.K)
            self.shard_finish()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_rank(rank, world, port, K, iters, out_q, fail_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise SystemExit(3)  # leaves before the first exchange
        h = FakeHandle(K)
        sh = SH.ShardedElf(h, rank=rank, world=world, device="cpu")
        sh.step(iters)
        out_q.put((rank, "ok", h.state.tobytes(), sh.exchanged_bytes))
    except SystemExit:
        raise
    except Exception as e:  # noqa: BLE001 - reported to the parent
        out_q.put((rank, "error", repr(e), 0))
    finally:
        if rank != fail_rank:
            try:
                dist.destroy_process_group()
            except Exception:  # noqa: BLE001
                pass


def _spawn(world, K, iters, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run_rank, args=(r, world, port, K, iters, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world - (1 if fail_rank >= 0 else 0)):
        r, status, payload, nbytes = q.get(timeout=120)
        res[r] = (status, payload, nbytes)
    for p in procs:
        p.join(timeout=60)
    return res


def test_led_blocks_partition():
    for K, W in ((49, 2), (225, 8), (3, 5), (1, 1), (16, 4)):
        b = SH.led_blocks(K, W)
        assert len(b) == W and b[0][0] == 0 and b[-1][1] == K
        assert all(x[1] == y[0] for x, y in zip(b, b[1:]))
        sizes = [k1 - k0 for k0, k1 in b]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        SH.led_blocks(4, 0)


@pytest.mark.parametrize("world,K", [(2, 49), (3, 10), (3, 2)])
def test_sharded_state_equals_one_process(world, K):
    """Every rank ends bitwise where one process running all LEDs ends (K = 2 on 3 ranks leaves
    one rank without LEDs)."""
    ref = FakeHandle(K)
    ref.step(4)
    res = _spawn(world, K, 4)
    row = FakeHandle(K).shard_row_floats()
    bmax = max(k1 - k0 for k0, k1 in SH.led_blocks(K, world))
    for r in range(world):
        status, payload, nbytes = res[r]
        assert status == "ok", payload
        assert np.frombuffer(payload, np.float32).tobytes() == ref.state.tobytes()
        assert nbytes == 4 * world * bmax * row * 4   # 4 iterations of [world, bmax * row] float32


def test_a_rank_that_leaves_before_the_exchange_fails_the_others():
    """Failure detection on the host: rank 1 exits before the first exchange; rank 0's exchange
    must end with an error (gloo reports the closed peer or the group's timeout) instead of hanging."""
    res = _spawn(2, 8, 2, fail_rank=1)
    status, payload, _ = res[0]
    assert status == "error", payload
