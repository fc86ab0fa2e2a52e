"""Serving form: the continuous-batching server (csrc/server.cu).

A mix of problem shapes arrives while earlier jobs are still on the GPU; every
result must equal the one-at-a-time plain path bit for bit (each job's
arithmetic is that of a lone run; nothing is shared between jobs), also when a
tight memory budget forces requests to wait and idle handles to be evicted.
"""
import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E
from paper_2209_14671_gb300 import serve as S

pytestmark = pytest.mark.gpu


def _request(n, u, grid, step, na_px, seed, n_iter):
    dk = 1.0 / n
    c = (np.arange(grid) - (grid - 1) // 2) * step
    cy, cx = np.meshgrid(c, c, indexing="ij")
    k_xy = np.stack([cx.ravel() * dk, cy.ravel() * dk], axis=1)
    geo = O.make_geometry(n, u, k_xy, na_px * dk, 1.0, 1.0)
    N = n * u
    g = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    obj = (0.6 + 0.3 * np.cos(2 * np.pi * (xx + seed) / N)) * np.exp(0.4j * np.sin(2 * np.pi * (yy + 2 * xx) / N))
    I = O.forward_intensity(O.spectrum_from_object(obj), geo.support.astype(complex), geo)
    I = np.ascontiguousarray((I + 1e-3 * g.standard_normal(I.shape)).astype(np.float32))
    return dict(n=n, u=u, k_xy=k_xy.astype(np.float32), na=na_px * dk, wl=1.0, dx=1.0, I=I, n_iter=n_iter)


@pytest.fixture(scope="module")
def requests():
    B.build()
    E.load()
    shapes = [(32, 4, 3, 5, 7.5), (32, 4, 5, 5, 7.5), (64, 2, 5, 6, 12.0), (64, 4, 3, 8, 12.0)]
    reqs = []
    for i in range(20):
        n, u, grid, step, na_px = shapes[i % len(shapes)]
        reqs.append(_request(n, u, grid, step, na_px, seed=i, n_iter=6 + (i % 3) * 4))
    return reqs


def test_results_in_the_mix_equal_lone_runs(requests):
    _, _, lone = S.run_serial(requests)
    arrivals = np.linspace(0.0, 0.02, len(requests))
    with S.Server(budget_bytes=8 << 30, max_active=6) as srv:
        lat, makespan, mixed = S.run_stream(srv, requests, arrivals, collect=True)
        st = srv.stats()
    print(f"serving: {len(requests)} requests, makespan {makespan * 1e3:.1f} ms, "
          f"p50 {np.percentile(lat, 50) * 1e3:.2f} ms, p99 {np.percentile(lat, 99) * 1e3:.2f} ms, {st}")
    for i in range(len(requests)):
        assert np.array_equal(mixed[i], lone[i]), i
    assert st["active"] == 0 and st["queued"] == 0 and st["handles_created"] <= 6 * 4


def test_tight_budget_waits_and_evicts(requests):
    _, _, lone = S.run_serial(requests[:8])
    # room for about two of the handles: admission must wait and evict idle shapes
    with S.Server(budget_bytes=8 << 20, max_active=8) as srv:
        lat, _, mixed = S.run_stream(srv, requests[:8], np.zeros(8), collect=True)
        st = srv.stats()
    assert st["used_bytes"] <= 8 << 20
    assert st["handles_created"] > 4           # some shapes were evicted and created again
    for i in range(8):
        assert np.array_equal(mixed[i], lone[i]), i


def test_server_error_paths(requests):
    r = requests[0]
    with S.Server(budget_bytes=1 << 30, max_active=2) as srv:
        srv.submit(7, r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], r["I"], r["n_iter"])
        with pytest.raises(E.ElfError) as ei:
            srv.submit(7, r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], r["I"], r["n_iter"])
        assert ei.value.code == E.ELF_EINVAL
        with pytest.raises(E.ElfError) as ei:
            srv.result(7)                      # not finished yet (not even admitted)
        assert ei.value.code == E.ELF_ESTATE
        done = []
        while not done:
            done = srv.progress()
        assert done == [7]
        assert srv.result(7).shape == (r["n"] * r["u"],) * 2
    with S.Server(budget_bytes=1 << 20, max_active=2) as srv:
        with pytest.raises(E.ElfError) as ei:   # cannot fit even alone
            srv.submit(1, r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], r["I"], r["n_iter"])
        assert ei.value.code == E.ELF_ENOMEM
