"""Thin ctypes binding of the C ABI in include/elfpie.h (argument marshalling only).

Every step of the Elfpie iteration runs in libelfpie.so's CUDA kernels; this module
only converts Python / NumPy / torch arguments to plain pointers and sizes.  There
is no CPU fallback: ``load()`` raises if the in-tree library has not been built.

Arrays: NumPy arrays are host memory, torch CUDA tensors device memory (their
``data_ptr()``).  Complex arrays are complex64 (interleaved float pairs).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libelfpie.so")

ELF_OK, ELF_EINVAL, ELF_ENOMEM, ELF_ECUDA, ELF_ENUMERIC, ELF_ETIMEOUT, ELF_ESTATE = 0, -1, -2, -3, -4, -5, -6

c_int, c_double, c_float, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
P_float, P_double, P_int = ctypes.POINTER(c_float), ctypes.POINTER(c_double), ctypes.POINTER(c_int)


class ElfProblem(ctypes.Structure):
    _fields_ = [("n_lowres", c_int), ("upsample", c_int), ("n_led", c_int), ("k_xy", P_float),
                ("na", c_double), ("wavelength_um", c_double), ("pixel_um", c_double), ("n_mux", c_int)]


class ElfOptions(ctypes.Structure):
    _fields_ = [("fidelity", c_int), ("omega_iso", c_int), ("learn_pupil", c_int), ("pupil_filter", c_int),
                ("alpha", c_double), ("beta", c_double), ("gamma1", c_double), ("gamma2", c_double),
                ("s0_psi", c_double), ("s0_pupil", c_double), ("eta_opt", c_double), ("eta_h", c_double),
                ("tau_fid", c_double), ("tau_h", c_double), ("tile_dft", c_int), ("g_exponent", c_double),
                ("tile_path", c_int)]


class ElfDegradeParams(ctypes.Structure):
    _fields_ = [("illum_c", c_double), ("waist_px", c_double), ("gauss_a", c_double), ("snp_density", c_double)]


class ElfState(ctypes.Structure):
    _fields_ = [("psi", P_float), ("mu_psi", P_float), ("v_psi", P_float), ("delta_psi", P_float),
                ("pupil", P_float), ("mu_pupil", P_float), ("v_pupil", P_float), ("delta_pupil", P_float),
                ("t", c_int), ("alpha", c_double), ("beta", c_double)]


# name -> (restype, argtypes): every symbol declared in include/elfpie.h
SIGNATURES = {
    "elf_default_options": (c_int, [ctypes.POINTER(ElfOptions)]),
    "elf_create": (c_int, [ctypes.POINTER(ElfProblem), ctypes.POINTER(ElfOptions), c_void_p, ctypes.POINTER(c_void_p)]),
    "elf_set_measurements": (c_int, [c_void_p, c_void_p, c_int]),
    "elf_step": (c_int, [c_void_p, c_int]),
    "elf_get_object": (c_int, [c_void_p, c_void_p, c_int]),
    "elf_get_pupil": (c_int, [c_void_p, c_void_p, c_int]),
    "elf_get_spectrum": (c_int, [c_void_p, c_void_p, c_int]),
    "elf_get_costs": (c_int, [c_void_p, P_double, c_int]),
    "elf_get_norms": (c_int, [c_void_p, P_double, c_int]),
    "elf_selftest_wait_timeout": (c_int, [c_void_p, ctypes.c_longlong, P_double]),
    "elf_get_state": (c_int, [c_void_p, ctypes.POINTER(ElfState), c_int]),
    "elf_set_state": (c_int, [c_void_p, ctypes.POINTER(ElfState), c_int]),
    "elf_cost_grad": (c_int, [c_void_p, c_void_p, c_void_p, P_double, c_void_p, c_void_p, c_int]),
    "elf_simulate": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "elf_get_tile_grads": (c_int, [c_void_p, c_void_p, c_int]),
    "elf_get_support": (c_int, [c_void_p, P_int]),
    "elf_get_weights": (c_int, [c_void_p, P_double, P_double]),
    "elf_set_tracing": (c_int, [c_void_p, c_int]),
    "elf_get_stage_times": (c_int, [c_void_p, P_float, c_int]),
    "elf_get_stage_spans": (c_int, [c_void_p, P_float, c_int]),
    "elf_graph_kernel_count": (c_int, [c_void_p]),
    "elf_server_create": (c_int, [ctypes.c_size_t, c_int, ctypes.POINTER(c_void_p)]),
    "elf_server_submit": (c_int, [c_void_p, ctypes.POINTER(ElfProblem), ctypes.POINTER(ElfOptions), c_void_p, c_int,
                                  ctypes.c_longlong]),
    "elf_server_progress": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_longlong), c_int, ctypes.POINTER(c_int)]),
    "elf_server_result": (c_int, [c_void_p, ctypes.c_longlong, c_void_p]),
    "elf_server_cancel": (c_int, [c_void_p, ctypes.c_longlong]),
    "elf_server_stats": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "elf_server_destroy": (None, [c_void_p]),
    "elf_estimate_weights_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "elf_degrade": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                            ctypes.POINTER(ElfDegradeParams), c_void_p]),
    "elf_noise_level": (c_int, [c_void_p, c_void_p, c_void_p, P_double]),
    "elf_lsnr": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_void_p, P_double]),
    "elf_object_quality": (c_int, [c_void_p, c_void_p, P_double]),
    "elf_measure_fp32_peak": (c_int, [c_int, c_int, c_void_p, P_double, P_double]),
    "elf_shard_row_floats": (c_int, [c_void_p]),
    "elf_shard_tiles": (c_int, [c_void_p, c_int, c_int]),
    "elf_shard_export": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "elf_shard_import": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "elf_shard_finish": (c_int, [c_void_p]),
    "elf_destroy": (None, [c_void_p]),
    "elf_strerror": (ctypes.c_char_p, [c_int]),
    "elf_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libelfpie.so (built in-tree by ``build.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libelfpie.so not found at {path}: run paper_2209_14671_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ElfError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = f"{where}: {lib.elf_strerror(code).decode()} ({code}): {lib.elf_last_error().decode()}"
        super().__init__(msg)
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise ElfError(rc, where)
    return rc


def _ptr(x):
    """(pointer, is_device) of a NumPy array or torch tensor (must be contiguous)."""
    if x is None:
        return None, 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    raise TypeError(f"unsupported array type {type(x)}")


def _dev_ptr(x) -> int:
    """Device address of a contiguous CUDA tensor (0 for None); the evaluation calls take device memory."""
    if x is None:
        return 0
    p, dev = _ptr(x)
    if not dev:
        raise ValueError("the evaluation calls take CUDA tensors")
    return p


def lsnr(rec, truth, stream=None) -> float:
    """LSNR of Eq. 22 (dB) of two contiguous float32 CUDA tensors of equal size."""
    if rec.numel() != truth.numel():
        raise ValueError("rec and truth differ in size")
    v = c_double()
    _check(load().elf_lsnr(c_void_p(_dev_ptr(rec)), c_void_p(_dev_ptr(truth)), int(rec.numel()),
                           c_void_p(_stream_handle(stream)), ctypes.byref(v)), "elf_lsnr")
    return v.value


def default_options(**overrides) -> ElfOptions:
    o = ElfOptions()
    _check(load().elf_default_options(ctypes.byref(o)), "elf_default_options")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Elf:
    """One reconstruction problem held on the GPU (an ``elf_handle``)."""

    def __init__(self, n, upsample, k_xy, na, wavelength_um, pixel_um, options=None, stream=None, mux=1):
        lib = load()
        k = np.ascontiguousarray(np.asarray(k_xy, dtype=np.float32).reshape(-1, 2))
        self._k = k
        prob = ElfProblem(int(n), int(upsample), int(k.shape[0]), k.ctypes.data_as(P_float),
                          float(na), float(wavelength_um), float(pixel_um), int(mux))
        if options is None:
            options = default_options()
        elif isinstance(options, dict):
            options = default_options(**options)
        self.options = options
        h = c_void_p()
        _check(lib.elf_create(ctypes.byref(prob), ctypes.byref(options), c_void_p(_stream_handle(stream)),
                              ctypes.byref(h)), "elf_create")
        self._h = h
        self.n, self.u, self.K = int(n), int(upsample), int(k.shape[0])
        self.mux = int(mux) if int(mux) > 0 else 1
        self.n_img = self.K // self.mux  # measured images (Eq. 1)
        self.N = self.n * self.u
        self.S = _check(lib.elf_get_support(self._h, None), "elf_get_support")

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().elf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ calls
    def set_measurements(self, I):
        p, dev = _ptr(I)
        _check(load().elf_set_measurements(self._h, c_void_p(p), dev), "elf_set_measurements")

    def step(self, n_iter: int = 1):
        _check(load().elf_step(self._h, int(n_iter)), "elf_step")

    # ------------------------------------------------------------ LED sharding of one iteration
    def shard_row_floats(self) -> int:
        return _check(load().elf_shard_row_floats(self._h), "elf_shard_row_floats")

    def shard_tiles(self, led_begin: int, led_end: int):
        _check(load().elf_shard_tiles(self._h, int(led_begin), int(led_end)), "elf_shard_tiles")

    def shard_export(self, led_begin: int, led_end: int, out):
        p, dev = _ptr(out)
        _check(load().elf_shard_export(self._h, int(led_begin), int(led_end), c_void_p(p), dev), "elf_shard_export")
        return out

    def shard_import(self, led_begin: int, led_end: int, src):
        p, dev = _ptr(src)
        _check(load().elf_shard_import(self._h, int(led_begin), int(led_end), c_void_p(p), dev), "elf_shard_import")

    def shard_finish(self):
        _check(load().elf_shard_finish(self._h), "elf_shard_finish")

    def _get(self, fn, shape, out):
        if out is None:
            out = np.empty(shape, dtype=np.complex64)
        p, dev = _ptr(out)
        _check(fn(self._h, c_void_p(p), dev), fn.__name__)
        return out

    def get_object(self, out=None):
        return self._get(load().elf_get_object, (self.N, self.N), out)

    def get_spectrum(self, out=None):
        return self._get(load().elf_get_spectrum, (self.N, self.N), out)

    def get_pupil(self, out=None):
        return self._get(load().elf_get_pupil, (self.n, self.n), out)

    def get_tile_grads(self, out=None):
        return self._get(load().elf_get_tile_grads, (self.K, self.S), out)

    def get_support(self) -> np.ndarray:
        idx = np.empty(self.S, dtype=np.int32)
        _check(load().elf_get_support(self._h, idx.ctypes.data_as(P_int)), "elf_get_support")
        return idx

    def get_costs(self, max_iter: int = 4096) -> np.ndarray:
        out = np.zeros((max_iter, 3), dtype=np.float64)
        cnt = _check(load().elf_get_costs(self._h, out.ctypes.data_as(P_double), int(max_iter)), "elf_get_costs")
        return out[:cnt]

    def get_norms(self, max_iter: int = 4096) -> np.ndarray:
        """[count][2] FP64 (||g||, ||Delta Psi||) per iteration, oldest first."""
        out = np.zeros((max_iter, 2), dtype=np.float64)
        cnt = _check(load().elf_get_norms(self._h, out.ctypes.data_as(P_double), int(max_iter)), "elf_get_norms")
        return out[:cnt]

    def selftest_wait_timeout(self, limit: int) -> float:
        """Runs the bounded-wait failure path (see elf_selftest_wait_timeout); returns its ms."""
        ms = c_double()
        _check(load().elf_selftest_wait_timeout(self._h, int(limit), ctypes.byref(ms)), "elf_selftest_wait_timeout")
        return ms.value

    def get_weights(self):
        a, b = c_double(), c_double()
        _check(load().elf_get_weights(self._h, ctypes.byref(a), ctypes.byref(b)), "elf_get_weights")
        return a.value, b.value

    def _state_struct(self, arrays, t=0, alpha=0.0, beta=0.0):
        ptrs = []
        dev = 0
        for a in arrays:
            p, dev = _ptr(a)
            ptrs.append(ctypes.cast(c_void_p(p), P_float))
        return ElfState(*ptrs, int(t), float(alpha), float(beta)), dev

    def get_state(self) -> dict:
        N, n = self.N, self.n
        arrs = [np.empty((N, N), np.complex64), np.empty((N, N), np.complex64), np.empty((N, N), np.float32),
                np.empty((N, N), np.float32), np.empty((n, n), np.complex64), np.empty((n, n), np.complex64),
                np.empty((n, n), np.float32), np.empty((n, n), np.float32)]
        st, dev = self._state_struct(arrs)
        _check(load().elf_get_state(self._h, ctypes.byref(st), dev), "elf_get_state")
        keys = ["psi", "mu_psi", "v_psi", "delta_psi", "pupil", "mu_p", "v_p", "delta_p"]
        out = dict(zip(keys, arrs))
        out.update(t=st.t, alpha=st.alpha, beta=st.beta)
        return out

    def set_state(self, psi, mu_psi, v_psi, delta_psi, pupil, mu_p, v_p, delta_p, t, alpha, beta):
        arrs = [np.ascontiguousarray(psi, np.complex64), np.ascontiguousarray(mu_psi, np.complex64),
                np.ascontiguousarray(v_psi, np.float32), np.ascontiguousarray(delta_psi, np.float32),
                np.ascontiguousarray(pupil, np.complex64), np.ascontiguousarray(mu_p, np.complex64),
                np.ascontiguousarray(v_p, np.float32), np.ascontiguousarray(delta_p, np.float32)]
        st, dev = self._state_struct(arrs, t, alpha, beta)
        _check(load().elf_set_state(self._h, ctypes.byref(st), dev), "elf_set_state")

    def cost_grad(self, psi, pupil, g_psi=None, g_pupil=None):
        """(costs float64 [L_fid, L_A, L_Phi, L], g_psi, g_pupil) at (psi, pupil), L the Eq. 8 total
        summed by the library; outputs allocated as NumPy if None."""
        if g_psi is None:
            g_psi = np.empty((self.N, self.N), np.complex64)
        if g_pupil is None:
            g_pupil = np.empty((self.n, self.n), np.complex64)
        c = (c_double * 4)()
        pp, dev = _ptr(psi)
        pq, _ = _ptr(pupil)
        gp, _ = _ptr(g_psi)
        gq, _ = _ptr(g_pupil)
        _check(load().elf_cost_grad(self._h, c_void_p(pp), c_void_p(pq), c, c_void_p(gp), c_void_p(gq), dev),
               "elf_cost_grad")
        return np.array(c[:], dtype=np.float64), g_psi, g_pupil

    STAGES = ("iteration", "tile", "hessian", "pupil_grad", "gather_update", "pupil_update", "cost")

    def set_tracing(self, enable: bool = True):
        _check(load().elf_set_tracing(self._h, int(bool(enable))), "elf_set_tracing")

    def stage_times(self) -> dict:
        """{stage: ms} of the most recent traced iteration (synchronises)."""
        ms = (c_float * len(self.STAGES))()
        cnt = _check(load().elf_get_stage_times(self._h, ms, len(self.STAGES)), "elf_get_stage_times")
        return {self.STAGES[i]: float(ms[i]) for i in range(cnt)}

    def stage_spans(self) -> dict:
        """{stage: (start_ms, end_ms)} from the start of the most recent traced iteration (synchronises)."""
        sp = (c_float * (2 * len(self.STAGES)))()
        cnt = _check(load().elf_get_stage_spans(self._h, sp, len(self.STAGES)), "elf_get_stage_spans")
        return {self.STAGES[i]: (float(sp[2 * i]), float(sp[2 * i + 1])) for i in range(cnt)}

    def kernels_per_step(self) -> int:
        return _check(load().elf_graph_kernel_count(self._h), "elf_graph_kernel_count")

    # ------------------------------------------------------------ evaluation (Sec. 4.1)
    def degrade(self, I_clean, out, c=0.0, waist_px=15.0, zeta=None, background=None, gauss_a=0.0, xi=None,
                snp_density=0.0, u_snp=None):
        """Eqs. 2 / 20 on device tensors [K/M, n, n] (background [K/M]) into ``out``."""
        prm = ElfDegradeParams(float(c), float(waist_px), float(gauss_a), float(snp_density))
        ptrs = [_dev_ptr(x) for x in (I_clean, zeta, background, xi, u_snp, out)]
        _check(load().elf_degrade(self._h, *[c_void_p(p) for p in ptrs[:5]], ctypes.byref(prm), c_void_p(ptrs[5])),
               "elf_degrade")
        return out

    def noise_level(self, I_sim, I_noised) -> float:
        """NL of Eq. 21 (percent) of two device tensors [K/M, n, n] over the dark-field images."""
        v = c_double()
        _check(load().elf_noise_level(self._h, c_void_p(_dev_ptr(I_sim)), c_void_p(_dev_ptr(I_noised)),
                                      ctypes.byref(v)), "elf_noise_level")
        return v.value

    def object_quality(self, obj_true):
        """(amplitude LSNR, phase LSNR) of Eq. 22 of the current object against a device complex64
        tensor [N, N], after the least-squares global phase."""
        out = (c_double * 2)()
        _check(load().elf_object_quality(self._h, c_void_p(_dev_ptr(obj_true)), out), "elf_object_quality")
        return out[0], out[1]

    def simulate(self, obj, out=None):
        """Predicted intensities of Eq. 1 [K/M, n, n] float32 of the spatial object ``obj``
        (|o_n|^2 per LED when M = 1, the sum over each image's M LEDs otherwise)."""
        if out is None:
            out = np.empty((self.n_img, self.n, self.n), np.float32)
        po, dev = _ptr(obj)
        pi, dev2 = _ptr(out)
        _check(load().elf_simulate(self._h, c_void_p(po), c_void_p(pi), dev2), "elf_simulate")
        return out


def estimate_weights_noalloc(I_dev, n_led: int, n_lowres: int, fidelity: int, weights_dev, stream=None):
    """Eq. 16/17 alpha = beta into ``weights_dev`` (device, 2 float64) without any device
    allocation, for callers that cannot allocate; asynchronous on ``stream``."""
    pi, dev_i = _ptr(I_dev)
    pw, dev_w = _ptr(weights_dev)
    if not (dev_i and dev_w):
        raise ValueError("I and weights must be device tensors")
    _check(load().elf_estimate_weights_noalloc(c_void_p(pi), int(n_led), int(n_lowres), int(fidelity),
                                               c_void_p(pw), c_void_p(_stream_handle(stream))),
           "elf_estimate_weights_noalloc")


def measure_fp32_peak(iters: int = 32768, repeats: int = 5, stream=None) -> tuple[float, float]:
    """(TFLOP/s, ms) of the best of `repeats` launches of the library's FP32 FMA-throughput kernel on
    the current device (synchronises)."""
    tf = c_double()
    ms = c_double()
    _check(load().elf_measure_fp32_peak(int(iters), int(repeats), c_void_p(_stream_handle(stream)), ctypes.byref(tf),
                                        ctypes.byref(ms)), "elf_measure_fp32_peak")
    return float(tf.value), float(ms.value)


def exported_symbols_from_header(header_path: str) -> list[str]:
    """Names of the functions declared in include/elfpie.h (for the load test)."""
    import re
    text = open(header_path).read()
    return sorted(set(re.findall(r"\b(elf_[a-z_]+)\s*\(", text)))
