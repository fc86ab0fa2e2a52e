"""All-cores driver of the FP64 oracle (TEST INFRASTRUCTURE: used by ``tests/`` and by
``bench.py``'s CPU-baseline and reference legs, never by the CUDA product path).

The per-LED terms of Eqs. 9-11 and 18 are independent (Sec. 3.4), so the LEDs are
split into contiguous blocks, one per worker process; each worker runs the oracle's
own ``fidelity_cost_grad`` on its block and leaves its partial sums of L_fid,
dL/d(conj Psi) and dL/d(conj P) in shared memory, and the caller adds the blocks in
block order.  Meanwhile the calling process evaluates the Hessian branch
(``hessian_cost_grad``) and then applies the same composition as
``elfpie_oracle.iteration`` (it is that function, given this fidelity evaluator).
Nothing of the method's arithmetic lives here: only the partition, the shared
buffers and the block-order sum.

Workers are started with the ``spawn`` method (no fork of a process that may hold a
CUDA context).  Multiplexed problems (M > 1) keep their images whole: blocks are
made of whole images.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import elfpie_oracle as O

_W = {}  # per worker process: shared arrays and the geometry of its block


def _attach(name, shape, dtype):
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _worker_init(spec):
    geo = spec["geo"]
    _W["spec"] = spec
    _W["shm"] = []
    for key, shape, dtype in (("psi", (geo.N, geo.N), np.complex128), ("pupil", (geo.n, geo.n), np.complex128),
                              ("I", (geo.n_images, geo.n, geo.n), np.float64),
                              ("gpsi", (spec["blocks"], geo.N, geo.N), np.complex128),
                              ("gp", (spec["blocks"], geo.n, geo.n), np.complex128)):
        shm, arr = _attach(spec["names"][key], shape, dtype)
        _W["shm"].append(shm)
        _W[key] = arr


def _worker_block(job):
    b, opt = job
    spec = _W["spec"]
    geo = spec["geo"]
    i0, i1 = spec["image_ranges"][b]
    sub = O.Geometry(n=geo.n, u=geo.u, N=geo.N, dk=geo.dk, offsets=geo.offsets[i0 * geo.mux:i1 * geo.mux],
                     origins=geo.origins[i0 * geo.mux:i1 * geo.mux], support=geo.support, mux=geo.mux)
    cost, g_psi, g_p, _ = O.fidelity_cost_grad(_W["psi"], _W["pupil"], _W["I"][i0:i1], sub, opt)
    _W["gpsi"][b] = g_psi
    _W["gp"][b] = g_p
    return cost


def image_blocks(n_images: int, blocks: int):
    """Contiguous, near-equal [i0, i1) ranges of images, in order (the first ones one longer)."""
    blocks = max(1, min(blocks, n_images))
    q, r = divmod(n_images, blocks)
    out, i0 = [], 0
    for b in range(blocks):
        i1 = i0 + q + (1 if b < r else 0)
        out.append((i0, i1))
        i0 = i1
    return out


class ParallelOracle:
    """Process pool over LED blocks for one problem (geometry and measurements fixed).

    ``po.fidelity`` has the signature of ``fidelity_cost_grad`` (tiles are not
    supported) and returns a callable that waits for the blocks, so that
    ``O.iteration(..., fidelity=po.fidelity)`` overlaps the Hessian branch with them.
    """

    def __init__(self, geo: O.Geometry, I, workers: int | None = None):
        workers = workers or max(1, (os.cpu_count() or 2) - 1)
        self.geo = geo
        self.ranges = image_blocks(geo.n_images, workers)
        self.blocks = len(self.ranges)
        self.cores = self.blocks + 1  # the workers and the calling process (Hessian branch)
        N, n = geo.N, geo.n
        sizes = {"psi": N * N * 16, "pupil": n * n * 16, "I": geo.n_images * n * n * 8,
                 "gpsi": self.blocks * N * N * 16, "gp": self.blocks * n * n * 16}
        self._shm = {k: shared_memory.SharedMemory(create=True, size=max(v, 16)) for k, v in sizes.items()}
        self.psi = np.ndarray((N, N), np.complex128, buffer=self._shm["psi"].buf)
        self.pupil = np.ndarray((n, n), np.complex128, buffer=self._shm["pupil"].buf)
        self.I = np.ndarray((geo.n_images, n, n), np.float64, buffer=self._shm["I"].buf)
        self.gpsi = np.ndarray((self.blocks, N, N), np.complex128, buffer=self._shm["gpsi"].buf)
        self.gp = np.ndarray((self.blocks, n, n), np.complex128, buffer=self._shm["gp"].buf)
        self.I[...] = np.asarray(I, dtype=np.float64)
        spec = {"geo": geo, "blocks": self.blocks, "image_ranges": self.ranges,
                "names": {k: v.name for k, v in self._shm.items()}}
        self._pool = mp.get_context("spawn").Pool(self.blocks, initializer=_worker_init, initargs=(spec,))

    def fidelity(self, psi, pupil, I, geo, opt, want_tiles=False):
        if want_tiles:
            raise ValueError("the parallel driver does not return per-LED tiles")
        if geo is not self.geo or I is not None and np.shape(I) != self.I.shape:
            raise ValueError("the parallel driver is bound to one geometry and one set of measurements")
        self.psi[...] = psi
        self.pupil[...] = pupil
        res = self._pool.map_async(_worker_block, [(b, opt) for b in range(self.blocks)])

        def finish():
            costs = res.get()
            cost = 0.0
            g_psi = np.zeros((geo.N, geo.N), dtype=np.complex128)
            g_p = np.zeros((geo.n, geo.n), dtype=np.complex128)
            for b in range(self.blocks):  # block order
                cost += costs[b]
                g_psi += self.gpsi[b]
                g_p += self.gp[b]
            return cost, g_psi, g_p, None
        return finish

    def run(self, state: O.State, opt: O.Options, n_iter: int):
        return O.run(state, self.I, self.geo, opt, n_iter, fidelity=self.fidelity)

    def close(self):
        if self._pool is not None:
            self._pool.terminate()
            self._pool.join()
            self._pool = None
        for shm in self._shm.values():
            shm.close()
            shm.unlink()
        self._shm = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
