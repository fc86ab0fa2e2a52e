"""Serving form: the continuous-batching server (csrc/server.cu).

A mix of problem shapes arrives while earlier jobs are still on the GPU; every
result must equal the one-at-a-time plain path bit for bit (each job's
arithmetic is that of a lone run; nothing is shared between jobs), also when a
tight memory budget forces requests to wait and idle handles to be evicted.
At the serving workload's own shapes (n 64/128/256, K 49/121/225) every served
result is also compared with the FP64 oracle, and the mixed stream must finish
sooner than the same jobs one at a time.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E
from paper_2209_14671_gb300 import inputs as IN
from paper_2209_14671_gb300 import serve as S

from _cases import rel

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


# ------------------------------------------------------------------ the serving workload's own shapes
CONFIG4 = [(n, g) for n in (64, 128, 256) for g in (7, 11, 15)]  # n x LED grid (K = 49, 121, 225)
ORACLE_ITERS = 4


def _config4_request(n, grid, seed, n_iter, options=None):
    """A request of the serving workload: workload-0 optics with an n x n camera and a grid x grid
    LED array, a seeded smooth object, measurements from the oracle's forward model at the true
    LED positions plus the workload's Gaussian noise (sigma 1e-3)."""
    w = IN.problem(0, grid=grid, n=n)
    geo_true = O.make_geometry(n, w["u"], w["k_xy_true"], w["na"], w["wavelength_um"], w["pixel_um"])
    obj = IN.object_field(1000 + seed, w)
    I = O.forward_intensity(O.spectrum_from_object(obj), geo_true.support.astype(complex), geo_true)
    I = np.ascontiguousarray(IN.corrupt(I, 0, w))
    return dict(n=n, u=w["u"], k_xy=w["k_xy"].astype(np.float32), na=w["na"], wl=w["wavelength_um"],
                dx=w["pixel_um"], I=I, n_iter=n_iter, options=options, w=w)


def test_served_results_match_oracle_at_serving_shapes():
    """Every shape of the serving workload (n in {64, 128, 256} x K in {49, 121, 225}) served in one
    mixed stream; each served object is compared with the FP64 oracle's run of the same request
    (Algorithm 1 from the initial state) and with the lone run.

    These requests use beta = 0 (alpha automatic): from the initial state the object is real and
    Eq. 14's normaliser turns FP32 rounding noise in its zero phase into a step that no FP32 run
    shares with FP64 (tests/golden/fp32_spread_w0.json); without the phase term the served run
    must follow the oracle to the full-run bound 1e-4."""
    B.build()
    E.load()
    opts = dict(beta=0.0)
    reqs = [_config4_request(n, g, seed=i, n_iter=ORACLE_ITERS, options=opts) for i, (n, g) in enumerate(CONFIG4)]
    _, _, lone = S.run_serial(reqs)
    with S.Server(budget_bytes=16 << 30, max_active=16) as srv:
        _, _, mixed = S.run_stream(srv, reqs, np.zeros(len(reqs)), collect=True)
    for i in range(len(reqs)):
        assert np.array_equal(mixed[i], lone[i]), i
    for i, r in enumerate(reqs):
        w = r["w"]
        geo = O.make_geometry(r["n"], r["u"], w["k_xy"], r["na"], r["wl"], r["dx"])
        opt = O.Options(beta=0.0)
        I = r["I"].astype(np.float64)
        st = O.init_state(I, geo, w["k_xy"], opt)
        ref, _ = O.run(st, I, geo, opt, r["n_iter"])
        e = rel(mixed[i], O.object_from_spectrum(ref.psi))
        print(f"n={r['n']} K={geo.K}: served object vs FP64 oracle after {r['n_iter']} iterations {e:.2e}")
        assert e < 1e-4, (r["n"], geo.K, e)


def test_cancelled_requests_leave_the_others_intact(requests):
    """Injected host faults of the serving loop: a running request cancelled (its job is waited for
    and dropped), a queued one withdrawn, a finished uncollected one discarded, and an unknown tag
    rejected.  The other requests' results are bitwise their lone runs, and nothing stays queued
    or active."""
    reqs = requests[:6]
    _, _, lone = S.run_serial(reqs)
    with S.Server(budget_bytes=8 << 30, max_active=2) as srv:
        for i, r in enumerate(reqs):
            srv.submit(i, r["n"], r["u"], r["k_xy"], r["na"], r["wl"], r["dx"], r["I"], r["n_iter"], r.get("options"))
        done = set(srv.progress())
        st = srv.stats()
        assert st["active"] + len(done) == 2 and st["queued"] == 4
        running = [i for i in (0, 1) if i not in done]
        for i in running[:1]:
            srv.cancel(i)
        srv.cancel(4)
        with pytest.raises(E.ElfError) as ei:
            srv.cancel(99)
        assert ei.value.code == E.ELF_EINVAL
        gone = set(running[:1]) | {4}
        want = set(range(len(reqs))) - gone
        got = {}
        deadline = time.monotonic() + 60.0
        while not want <= done and time.monotonic() < deadline:
            done |= set(srv.progress())
        assert want <= done and not (gone & done)
        srv.cancel(5)  # finished, not collected
        for i in sorted(want - {5}):
            got[i] = srv.result(i)
        st = srv.stats()
    for i, res in got.items():
        assert np.array_equal(res, lone[i]), i
    assert st["active"] == 0 and st["queued"] == 0


def test_small_jobs_overlap_on_the_device():
    """Continuous batching of latency-bound jobs: 16 reconstructions of the serving workload's
    smallest shape (64 x 64 images, 49 LEDs, 50 iterations) submitted together finish well before
    the same jobs run one at a time (each alone leaves most of the GPU idle), with every result equal
    to its lone run.  Both paths are warmed first (pooled handles, captured graphs)."""
    B.build()
    E.load()
    reqs = [_config4_request(64, 7, seed=200 + i, n_iter=50) for i in range(16)]
    S.run_serial(reqs)
    serial_t, _, lone = S.run_serial(reqs)
    with S.Server(budget_bytes=16 << 30, max_active=16) as srv:
        S.run_stream(srv, reqs, np.zeros(len(reqs)))
        _, makespan, mixed = S.run_stream(srv, reqs, np.zeros(len(reqs)), collect=True)
    print(f"16 small jobs: makespan {makespan * 1e3:.2f} ms against {serial_t.sum() * 1e3:.2f} ms one at a time")
    for i in range(len(reqs)):
        assert np.array_equal(mixed[i], lone[i]), i
    assert makespan < 0.8 * serial_t.sum()
