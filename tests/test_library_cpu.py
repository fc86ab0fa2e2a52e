"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol
declared in include/elfpie.h, and host-side validation rejects invalid problems
before any CUDA call (so these run without a GPU)."""
import ctypes
import os

import numpy as np
import pytest

from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "elfpie.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def test_exports_every_declared_symbol(lib):
    names = E.exported_symbols_from_header(HEADER)
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
        assert name in E.SIGNATURES, f"binding lacks {name}"


def test_default_options_match_paper_defaults(lib):
    o = E.default_options()
    assert (o.gamma1, o.gamma2, o.s0_psi) == (0.9, 0.999, 1.0)
    assert o.alpha < 0 and o.beta < 0 and o.fidelity == 0 and o.omega_iso == 1 and o.g_exponent == 1.0


def _create(n=64, u=4, k=((0.0, 0.0),), na=0.1, wl=0.63, dx=1.625, **opts):
    lib = E.load()
    kk = np.ascontiguousarray(np.asarray(k, np.float32).reshape(-1, 2))
    prob = E.ElfProblem(n, u, kk.shape[0], kk.ctypes.data_as(E.P_float), na, wl, dx)
    o = E.default_options(**opts)
    h = ctypes.c_void_p()
    rc = lib.elf_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h))
    return rc, lib.elf_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(n=48), "n_lowres"),
    (dict(u=3), "upsample"),
    (dict(n=256, u=8), "upsample"),
    (dict(k=((1.0, 0.0),)), "crop window"),          # 104 px offset: window [200, 264) leaves [0, 256)
    (dict(na=-0.1), "na"),
    (dict(wl=0.0), "wavelength_um"),
    (dict(k=((float("nan"), 0.0),)), "non-finite"),
    (dict(gamma1=1.5), "invalid options"),
    (dict(n=64, tile_dft=1), "tile_dft"),            # the tensor-core tile path is for n = 128
])
def test_invalid_problems_are_rejected(lib, kw, needle):
    rc, msg = _create(**kw)
    assert rc == E.ELF_EINVAL, (rc, msg)
    assert needle in msg


def test_server_queue_and_cancel_on_the_host(lib):
    """Injected host faults of the serving API without the device: requests that are only queued
    (no progress call, so nothing is created on a GPU) are withdrawn by elf_server_cancel, a second
    cancel and an unknown tag are rejected, a request over the memory budget is refused, and the
    server is left empty."""
    from paper_2209_14671_gb300 import serve as S
    k = np.zeros((1, 2), np.float32)
    I = np.zeros((1, 64, 64), np.float32)
    with S.Server(budget_bytes=1 << 30, max_active=2) as srv:
        srv.submit(1, 64, 4, k, 0.1, 0.63, 1.625, I, 5)
        srv.submit(2, 64, 4, k, 0.1, 0.63, 1.625, I, 5)
        with pytest.raises(E.ElfError) as ei:
            srv.submit(2, 64, 4, k, 0.1, 0.63, 1.625, I, 5)
        assert ei.value.code == E.ELF_EINVAL
        assert srv.stats()["queued"] == 2
        srv.cancel(1)
        assert srv.stats()["queued"] == 1
        for tag in (1, 99):
            with pytest.raises(E.ElfError) as ei:
                srv.cancel(tag)
            assert ei.value.code == E.ELF_EINVAL
        srv.cancel(2)
        assert srv.stats() == dict(used_bytes=0, active=0, queued=0, handles_created=0)
    with S.Server(budget_bytes=1 << 20, max_active=1) as srv:
        with pytest.raises(E.ElfError) as ei:
            srv.submit(3, 256, 4, k, 0.1, 0.63, 1.625, np.zeros((1, 256, 256), np.float32), 5)
        assert ei.value.code == E.ELF_ENOMEM


def test_strerror_covers_all_codes(lib):
    for code in range(0, -7, -1):
        assert lib.elf_strerror(code).decode() != "unknown error"
