"""Evaluation of Sec. 4.1 on the GPU against the FP64 oracle, through the C ABI: the degradations
of Eqs. 2 / 20 with given random fields, NL (Eq. 21), LSNR (Eq. 22) and the phase-aligned
quality of a reconstruction.

Bounds: continuous values 1e-5 relative L2 (FP32 blur and arithmetic against FP64); the salt &
pepper decisions are taken in FP64 on both sides and must agree pixel for pixel; NL and LSNR to
1e-6 relative and 1e-3 dB.
"""
import numpy as np
import pytest

import oracle as O
from paper_2209_14671_gb300 import build as B
from paper_2209_14671_gb300 import elfpie as E

from _cases import case, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    E.load()


def _elf(c, mux=1):
    return E.Elf(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], mux=mux)


def _fields(shape, seed):
    g = np.random.default_rng(seed)
    return dict(zeta=g.standard_normal(shape), xi=g.standard_normal(shape), u=g.random(shape),
                bg=g.uniform(0.0, 0.1, shape[0]))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name,mux,terms", [
    ("tiny16", 1, dict(c=0.3, waist_px=3.0, gauss_a=1e-2, snp_density=0.0625, background=True)),
    ("small32", 5, dict(c=0.5, waist_px=6.0, gauss_a=0.0, snp_density=0.0, background=False)),
    ("w0", 1, dict(c=0.0, gauss_a=1e-3, snp_density=0.05, background=True)),
    ("w0", 1, dict(c=0.2, waist_px=15.0, gauss_a=0.0, snp_density=0.0, background=False)),
])
def test_degrade_matches_oracle(name, mux, terms):
    c = case(name)
    geo = O.make_geometry(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], mux=mux)
    I0 = O.forward_intensity(O.spectrum_from_object(c["obj"]), geo.support.astype(complex), geo)
    I0 = I0.astype(np.float32).astype(np.float64)
    f = _fields(I0.shape, 91 + mux)
    for k in ("zeta", "xi", "u"):
        f[k] = f[k].astype(np.float32).astype(np.float64)
    f["bg"] = f["bg"].astype(np.float32).astype(np.float64)
    bg = f["bg"] if terms["background"] else None
    ref = O.degrade(I0, c=terms["c"], waist_px=terms.get("waist_px", 15.0), zeta=f["zeta"], background=bg,
                    gauss_a=terms["gauss_a"], xi=f["xi"], snp_density=terms["snp_density"], u_snp=f["u"])
    out = torch.empty(I0.shape, dtype=torch.float32, device="cuda")
    with _elf(c, mux) as elf:
        elf.degrade(_dev(I0), out, c=terms["c"], waist_px=terms.get("waist_px", 15.0), zeta=_dev(f["zeta"]),
                    background=_dev(bg) if bg is not None else None, gauss_a=terms["gauss_a"], xi=_dev(f["xi"]),
                    snp_density=terms["snp_density"], u_snp=_dev(f["u"]))
    got = out.cpu().numpy().astype(np.float64)
    d = terms["snp_density"]
    if d:
        hit = f["u"] < d
        assert np.array_equal(got[hit], ref[hit]) and hit.any()
    e = rel(got, ref)
    print(name, mux, terms, f"degrade {e:.2e}")
    assert e < 1e-5


@pytest.mark.parametrize("name,mux", [("w0", 1), ("small32", 5), ("tiny16", 3)])
def test_noise_level_matches_oracle(name, mux):
    c = case(name)
    geo = O.make_geometry(c["n"], c["u"], c["k_xy"], c["na"], c["wl"], c["dx"], mux=mux)
    I0 = O.forward_intensity(O.spectrum_from_object(c["obj"]), geo.support.astype(complex), geo).astype(np.float32)
    In = (I0 + 1e-2 * np.random.default_rng(92).standard_normal(I0.shape)).astype(np.float32)
    dark = O.darkfield_images(geo, c["na"], c["wl"])
    ref = O.noise_level(I0, In, dark)
    with _elf(c, mux) as elf:
        got = elf.noise_level(_dev(I0), _dev(In))
    print(name, mux, int(dark.sum()), "dark images", f"NL {got:.6f} vs {ref:.6f}")
    assert abs(got - ref) <= 1e-6 * max(abs(ref), 1e-12)


@pytest.mark.parametrize("count", [1, 7, 1000, 262144 + 13])
def test_lsnr_matches_oracle(count):
    g = np.random.default_rng(93 + count)
    truth = g.uniform(0.1, 1.0, count).astype(np.float32)
    rec = (truth + 0.02 * g.standard_normal(count) + 0.5).astype(np.float32)
    if count == 1:
        rec = np.array([truth[0] + 0.3], dtype=np.float32)  # b absorbs it: ||d - b|| = 0, infinite LSNR
    ref = O.lsnr(rec, truth) if count > 1 else float("inf")
    got = E.lsnr(_dev(rec), _dev(truth))
    print(count, got, ref)
    if count == 1:
        assert got == float("inf")
    else:
        assert abs(got - ref) < 1e-6 * abs(ref)


def test_object_quality_matches_oracle():
    c = case("w0")
    with _elf(c) as elf:
        elf.set_measurements(c["I"])
        elf.step(10)
        obj = elf.get_object()
        a, p = elf.object_quality(torch.from_numpy(c["obj"].astype(np.complex64)).cuda())
    ra, rp = O.object_quality(obj.astype(np.complex128), c["obj"].astype(np.complex64).astype(np.complex128))
    print(f"amplitude {a:.4f} / {ra:.4f} dB, phase {p:.4f} / {rp:.4f} dB")
    assert abs(a - ra) < 1e-3 and abs(p - rp) < 1e-3


def test_degrade_validates_its_arguments():
    c = case("tiny16")
    I0 = torch.zeros((9, 16, 16), dtype=torch.float32, device="cuda")
    out = torch.empty_like(I0)
    with _elf(c) as elf:
        for kw in (dict(c=0.5), dict(gauss_a=0.1), dict(snp_density=0.1), dict(c=1.5, zeta=I0),
                   dict(snp_density=-0.1, u_snp=I0), dict(c=0.5, zeta=I0, waist_px=0.0)):
            with pytest.raises(E.ElfError) as ei:
                elf.degrade(I0, out, **kw)
            assert ei.value.code == E.ELF_EINVAL
        with pytest.raises(E.ElfError) as ei:  # the output may not alias an input
            elf.degrade(I0, I0, gauss_a=0.1, xi=out)
        assert ei.value.code == E.ELF_EINVAL
