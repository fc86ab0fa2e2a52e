"""Serving form: continuous batching of many Elfpie reconstructions.

``Server`` is a thin binding of the C server (csrc/server.cu: memory admission,
pooled handles, one stream per job, non-blocking retirement).  ``run_stream``
replays a stream of requests with given arrival times against it and measures
each request's latency (arrival -> result on the host); ``run_serial`` runs the
same requests one at a time through the plain handle path for comparison.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import elfpie as E


class Server:
    def __init__(self, budget_bytes: int, max_active: int = 32):
        lib = E.load()
        h = ctypes.c_void_p()
        E._check(lib.elf_server_create(ctypes.c_size_t(int(budget_bytes)), int(max_active), ctypes.byref(h)),
                 "elf_server_create")
        self._h = h
        self._keep = {}       # tag -> (measurements, problem arrays) kept alive until collected
        self._done = (ctypes.c_longlong * 4096)()

    def submit(self, tag: int, n: int, u: int, k_xy, na: float, wavelength_um: float, pixel_um: float,
               I: np.ndarray, n_iter: int, options=None):
        k = np.ascontiguousarray(np.asarray(k_xy, np.float32).reshape(-1, 2))
        if not (isinstance(I, np.ndarray) and I.dtype == np.float32 and I.flags["C_CONTIGUOUS"]):
            raise TypeError("I must be a C-contiguous float32 array (pinned for asynchronous upload)")
        prob = E.ElfProblem(int(n), int(u), int(k.shape[0]), k.ctypes.data_as(E.P_float), float(na),
                            float(wavelength_um), float(pixel_um))
        opt = E.default_options(**(options or {}))
        E._check(E.load().elf_server_submit(self._h, ctypes.byref(prob), ctypes.byref(opt),
                                            ctypes.c_void_p(I.ctypes.data), int(n_iter), int(tag)),
                 "elf_server_submit")
        self._keep[int(tag)] = (I, k, n * u)

    def progress(self) -> list[int]:
        cnt = ctypes.c_int()
        E._check(E.load().elf_server_progress(self._h, self._done, len(self._done), ctypes.byref(cnt)),
                 "elf_server_progress")
        return [int(self._done[i]) for i in range(cnt.value)]

    def result(self, tag: int) -> np.ndarray:
        _, _, N = self._keep[int(tag)]
        out = np.empty((N, N), np.complex64)
        E._check(E.load().elf_server_result(self._h, int(tag), ctypes.c_void_p(out.ctypes.data)), "elf_server_result")
        del self._keep[int(tag)]
        return out

    def cancel(self, tag: int):
        """Withdraws a request (elf_server_cancel); its input buffer is released here."""
        E._check(E.load().elf_server_cancel(self._h, ctypes.c_longlong(int(tag))), "elf_server_cancel")
        self._keep.pop(int(tag), None)

    def stats(self) -> dict:
        used, act, q, created = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        E._check(E.load().elf_server_stats(self._h, ctypes.byref(used), ctypes.byref(act), ctypes.byref(q),
                                           ctypes.byref(created)), "elf_server_stats")
        return dict(used_bytes=used.value, active=act.value, queued=q.value, handles_created=created.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            E.load().elf_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_stream(server: Server, requests: list[dict], arrivals_s: np.ndarray, collect=None):
    """Submit requests[i] at arrivals_s[i] (seconds from start), poll until all are done.

    Each request dict: n, u, k_xy, na, wl, dx, I (pinned float32), n_iter, options.
    Returns (latencies_s, makespan_s, results dict if collect else None)."""
    order = np.argsort(arrivals_s, kind="stable")
    t0 = time.perf_counter()
    t_arr = {}
    lat = {}
    results = {} if collect else None
    nxt = 0
    pending = 0
    while nxt < len(order) or pending:
        now = time.perf_counter() - t0
        while nxt < len(order) and arrivals_s[order[nxt]] <= now:
            i = int(order[nxt])
            r = requests[i]
            server.submit(i, r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], r["I"], r["n_iter"],
                          r.get("options"))
            t_arr[i] = t0 + float(arrivals_s[i])
            nxt += 1
            pending += 1
        for tag in server.progress():
            t = time.perf_counter()
            lat[tag] = t - t_arr[tag]
            res = server.result(tag)
            if collect:
                results[tag] = res
            pending -= 1
    makespan = time.perf_counter() - t0
    return np.array([lat[i] for i in range(len(requests))]), makespan, results


def run_serial(requests: list[dict], stream=None):
    """The same jobs one at a time through the plain handle path (elf_set_measurements,
    elf_step, elf_get_object), handles created once per shape.  Returns
    (per-request service times in s, total time in s, results)."""
    handles = {}
    times, results = [], {}
    t_all = time.perf_counter()
    for i, r in enumerate(requests):
        key = (r["n"], r["u"], r["k_xy"].tobytes(), r["na"], r["wl"], r["dx"], repr(r.get("options")))
        if key not in handles:
            handles[key] = E.Elf(r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], options=r.get("options"),
                                 stream=stream)
        elf = handles[key]
        t = time.perf_counter()
        elf.set_measurements(r["I"])
        elf.step(r["n_iter"])
        results[i] = elf.get_object()
        times.append(time.perf_counter() - t)
    total = time.perf_counter() - t_all
    for h in handles.values():
        h.close()
    return np.array(times), total, results
