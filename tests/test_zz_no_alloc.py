"""The no-allocation weight estimate (elf_estimate_weights_noalloc).

Some callers cannot allocate device memory (their device memory belongs to
another allocator or a fixed budget, or their framework forbids allocations
while they run).  This entry point gives them the Eq. 16/17 weight without a
handle and without allocating; its scratch is a static device array.  These
tests call it through the C ABI and compare it with the weight the handle path
(elf_set_measurements) computes, on two calls in a row; they must pass alone in
a fresh process and after the other tests.  The file is named to be collected
last.
"""
import ctypes

import numpy as np
import pytest

from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E

from _cases import case

pytestmark = pytest.mark.gpu

TOL_ALPHA = 1e-6  # the tolerance the parity tests use for alpha


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    B.build()
    E.load()
    return torch, torch.device("cuda:0")


@pytest.mark.parametrize("name,fidelity", [("w0", 0), ("w0", 1), ("small32", 0)])
def test_noalloc_weights_match_handle_path_on_two_calls(torch_dev, name, fidelity):
    torch, dev = torch_dev
    c = case(name)
    with E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], options=dict(fidelity=fidelity)) as elf:
        elf.set_measurements(c["I"])
        a_ref, b_ref = elf.get_weights()
    I_dev = torch.from_numpy(c["I"]).to(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    K, n = c["I"].shape[0], c["I"].shape[1]
    for call in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize(dev)
        before = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
        E.estimate_weights_noalloc(I_dev, K, n, fidelity, out, stream)
        torch.cuda.synchronize(dev)
        after = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
        a, b = out.cpu().tolist()
        assert a == b
        assert abs(a - a_ref) <= TOL_ALPHA * abs(a_ref), (call, a, a_ref)
        if call == 1:
            # A coarse check of the claim itself: the first call may load the module, the second must
            # leave torch's allocator and the device's free memory (cudaMemGetInfo) exactly as they were.
            # It would not see an allocation freed again within the call.
            assert after == before, (before, after)


def test_noalloc_rejects_problems_beyond_the_static_scratch(torch_dev):
    torch, dev = torch_dev
    lib = E.load()
    dummy = torch.zeros(2, dtype=torch.float64, device=dev)
    # 20000 images of 256 x 256 need 20000 * 16 partials > ELF_NOALLOC_WEIGHT_MAX_PARTIALS
    rc = lib.elf_estimate_weights_noalloc(ctypes.c_void_p(dummy.data_ptr()), 20000, 256, 0,
                                          ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == E.ELF_EINVAL
    assert "too large for the static scratch" in lib.elf_last_error().decode()
    assert np.all(dummy.cpu().numpy() == 0)
