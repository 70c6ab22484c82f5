"""Python binding of libosar (ctypes, argument marshalling only).

Every step of the online SAR hot path runs in the library's CUDA kernels;
this module only converts NumPy arrays / torch tensors to pointers and status
codes to exceptions.  If the compiled library is missing the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libosar.so")

OSAR_OK, OSAR_E_INVALID, OSAR_E_OOM, OSAR_E_CUDA, OSAR_E_STATE, \
    OSAR_E_TIMEOUT, OSAR_E_NUMERIC, OSAR_E_IO = range(8)
OSAR_FP64, OSAR_FP32, OSAR_SPLIT_BF16 = 0, 1, 2
OSAR_DICT_IDENTITY, OSAR_DICT_HOST, OSAR_DICT_GAUSSIAN, OSAR_DICT_EDGELET = 0, 1, 2, 3
COPY_SLOTS = 4  # OSAR_COPY_SLOTS: osar_get_coeffs_async completion slots

PRECISIONS = {"fp64": OSAR_FP64, "fp32": OSAR_FP32, "split_bf16": OSAR_SPLIT_BF16}

KERNEL_CLASSES = {"phase": 0, "dict_gemm": 1, "gram_gemm": 2, "data_update": 3,
                  "matvec": 4, "fista_finalize": 5, "power_finalize": 6,
                  "block_term": 7, "dict_apply": 8}

# Symbols declared in include/osar.h (checked by the CPU test suite).
EXPORTS = [
    "osar_config_default", "osar_create", "osar_destroy", "osar_push_pulse",
    "osar_push_pulse_var",
    "osar_push_pulse_dev", "osar_iterate", "osar_get_coeffs",
    "osar_get_coeffs_dev", "osar_get_coeffs_async", "osar_wait_coeffs",
    "osar_get_lambda_state",
    "osar_get_state", "osar_get_dims", "osar_get_gram",
    "osar_get_gram_entries", "osar_get_b", "osar_gram_apply",
    "osar_gram_apply_static",
    "osar_simulate_pulse", "osar_unroll_grad", "osar_synchronize",
    "osar_get_metrics", "osar_set_lambda", "osar_set_gram_ahead",
    "osar_probe_bounded_wait", "osar_check_guards", "osar_poke_guard",
    "osar_batch_check_guards",
    "osar_profile_enable",
    "osar_profile_select",
    "osar_profile_sample",
    "osar_profile_ahead",
    "osar_profile_read", "osar_profile_reset", "osar_profile_passes",
    "osar_launch_count",
    "osar_device_bytes", "osar_save", "osar_load", "osar_last_error",
    "osar_version",
    "osar_batch_create", "osar_batch_destroy", "osar_batch_push",
    "osar_batch_iterate", "osar_batch_get_coeffs", "osar_batch_get_state",
    "osar_batch_autotune", "osar_batch_get_tuning", "osar_batch_info",
    "osar_batch_synchronize",
    "osar_batch_last_error",
]


class OsarConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("pixel_m", C.c_double),
        ("n_freq", C.c_int32), ("f_lo_hz", C.c_double), ("f_hi_hz", C.c_double),
        ("dict_kind", C.c_int32), ("n_atoms", C.c_int32),
        ("dict_c128", C.c_void_p), ("dict_seed", C.c_uint64),
        ("precision", C.c_int32),
        ("lam", C.c_double), ("lambda_relative", C.c_int32),
        ("power_iters_first", C.c_int32), ("power_iters", C.c_int32),
        ("lipschitz_margin", C.c_double),
        ("restart_momentum", C.c_int32), ("compensated", C.c_int32),
        ("cuda_stream", C.c_void_p),
        ("overlap_synthesis", C.c_int32), ("synth_ctas", C.c_int32),
        ("tc_pairs", C.c_int32), ("fuse_first_step", C.c_int32),
        ("n_lambdas", C.c_int32), ("lambda_list", C.c_void_p),
        ("defer_gram", C.c_int32), ("guard_bytes", C.c_int32),
        ("n_edgelet_lengths", C.c_int32), ("edgelet_lengths", C.c_void_p),
        ("n_edgelet_angles", C.c_int32), ("edgelet_angles_deg", C.c_void_p),
        ("fuse_power_gram", C.c_int32), ("pixel_gram", C.c_int32),
        ("gram_superblock", C.c_int32),
        ("gram_ahead", C.c_int32),
    ]


class OsarMetrics(C.Structure):
    _fields_ = [
        ("n_large", C.c_int32), ("n_nonzero", C.c_int32),
        ("n_support", C.c_int32), ("large_outside_support", C.c_int32),
        ("l1", C.c_double), ("max_abs", C.c_double),
        ("rms_signal", C.c_double), ("rms_noise", C.c_double),
        ("snr_db", C.c_double),
    ]


class OsarError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libosar status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libosar.so (built by paper_2603_08582_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"libosar.so not found at {path}; build it with "
            "`python -m paper_2603_08582_gb300.build` (needs nvcc)")
    lib = C.CDLL(path)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    I32 = C.c_int32
    sig = {
        "osar_config_default": (None, [C.POINTER(OsarConfig)]),
        "osar_create": (I32, [C.POINTER(OsarConfig), C.POINTER(P)]),
        "osar_destroy": (I32, [P]),
        "osar_push_pulse": (I32, [P, D, D]),
        "osar_push_pulse_dev": (I32, [P, D, P]),
        "osar_push_pulse_var": (I32, [P, D, D, D]),
        "osar_iterate": (I32, [P, I32, C.c_double, C.POINTER(I32)]),
        "osar_get_coeffs": (I32, [P, D]),
        "osar_get_coeffs_dev": (I32, [P, P]),
        "osar_get_coeffs_async": (I32, [P, D, I32]),
        "osar_wait_coeffs": (I32, [P, I32]),
        "osar_get_lambda_state": (I32, [P, I32, D, D, D, C.POINTER(I32)]),
        "osar_get_state": (I32, [P, C.POINTER(I32), D, D, D]),
        "osar_get_dims": (I32, [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]),
        "osar_get_gram": (I32, [P, D]),
        "osar_get_gram_entries": (I32, [P, C.POINTER(I32), C.POINTER(I32), I32, D]),
        "osar_get_b": (I32, [P, D]),
        "osar_gram_apply": (I32, [P, D, D]),
        "osar_gram_apply_static": (I32, [P, P, P]),
        "osar_simulate_pulse": (I32, [P, D, D, D]),
        "osar_unroll_grad": (I32, [P, I32, I32, C.c_double, C.c_double,
                                     C.c_double, D, D, D, D, D, D, D]),
        "osar_synchronize": (I32, [P]),
        "osar_set_lambda": (I32, [P, I32, C.c_double]),
        "osar_set_gram_ahead": (I32, [P, I32]),
        "osar_get_metrics": (I32, [P, C.c_double, C.POINTER(I32), I32,
                                   C.POINTER(OsarMetrics)]),
        "osar_probe_bounded_wait": (I32, [P, C.c_int64]),
        "osar_check_guards": (I32, [P, C.POINTER(I32)]),
        "osar_poke_guard": (I32, [P, I32]),
        "osar_batch_check_guards": (I32, [P, C.POINTER(I32)]),
        "osar_profile_enable": (I32, [P, I32]),
        "osar_profile_select": (I32, [P, C.c_uint32]),
        "osar_profile_sample": (I32, [P, I32, I32]),
        "osar_profile_ahead": (I32, [P, C.POINTER(C.c_int64), C.POINTER(I32)]),
        "osar_profile_read": (I32, [P, I32, C.POINTER(C.c_int64), D]),
        "osar_profile_reset": (I32, [P]),
        "osar_profile_passes": (I32, [P, C.POINTER(C.c_int64)]),
        "osar_launch_count": (I32, [P, C.POINTER(C.c_int64)]),
        "osar_device_bytes": (I32, [P, C.POINTER(C.c_int64)]),
        "osar_save": (I32, [P, C.c_char_p]),
        "osar_load": (I32, [C.c_char_p, C.POINTER(OsarConfig), C.POINTER(P)]),
        "osar_last_error": (C.c_char_p, [P]),
        "osar_version": (C.c_char_p, []),
        "osar_batch_create": (I32, [C.POINTER(OsarConfig), I32, P, C.POINTER(P)]),
        "osar_batch_destroy": (I32, [P]),
        "osar_batch_push": (I32, [P, C.POINTER(I32), D, D, I32]),
        "osar_batch_iterate": (I32, [P, I32, C.c_double, C.POINTER(I32)]),
        "osar_batch_get_coeffs": (I32, [P, I32, D]),
        "osar_batch_get_state": (I32, [P, I32, C.POINTER(I32), D, D, D]),
        "osar_batch_autotune": (I32, [P, C.POINTER(I32)]),
        "osar_batch_get_tuning": (I32, [P, C.POINTER(I32), C.POINTER(I32),
                                        C.POINTER(I32), D, D]),
        "osar_batch_info": (I32, [P, C.POINTER(I32), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64), C.POINTER(I32)]),
        "osar_batch_synchronize": (I32, [P]),
        "osar_batch_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def default_config() -> OsarConfig:
    cfg = OsarConfig()
    load_library().osar_config_default(C.byref(cfg))
    return cfg


def make_config(nx, ny, n_freq, f_lo_hz, f_hi_hz, pixel_m=1.0,
                precision="fp64", dictionary=None, n_atoms=None, dict_seed=0,
                lam=0.05, lambda_relative=True, power_iters_first=30,
                power_iters=4, lipschitz_margin=0.01, restart_momentum=False,
                compensated=True, stream=None, overlap_synthesis=True,
                synth_ctas=0, tc_pairs=3, fuse_first_step=True, lambdas=None,
                defer_gram=False, guard_bytes=0, edgelet_lengths=None,
                edgelet_angles=None, fuse_power_gram=True, pixel_gram=False,
                gram_superblock=0, gram_ahead=0):
    """Build an osar_config.  dictionary: None (identity), "gaussian"
    (seeded Philox atoms, needs n_atoms), "edgelet" (binary edgelets of
    edgelet_lengths x edgelet_angles degrees at every pixel) or an N x M
    complex array.  pixel_gram (edgelets only): keep the pixel-basis Gram
    P_n = sum F^H F and apply G_n = H^H P_n H instead of storing G_n;
    fuse_power_gram: form the pulse's first power step in the Gram update;
    gram_ahead: 0 in order, 1 the Gram update beside the previous burst when
    a model expects that to pay, 2 always (into a second Gram buffer)."""
    cfg = default_config()
    cfg.nx, cfg.ny, cfg.pixel_m = int(nx), int(ny), float(pixel_m)
    cfg.n_freq, cfg.f_lo_hz, cfg.f_hi_hz = int(n_freq), float(f_lo_hz), float(f_hi_hz)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    keep = None
    if dictionary is None:
        cfg.dict_kind = OSAR_DICT_IDENTITY
    elif isinstance(dictionary, str) and dictionary == "gaussian":
        cfg.dict_kind = OSAR_DICT_GAUSSIAN
        cfg.n_atoms = int(n_atoms)
        cfg.dict_seed = int(dict_seed)
    elif isinstance(dictionary, str) and dictionary == "edgelet":
        lv = np.ascontiguousarray(np.asarray(edgelet_lengths, dtype=np.int32))
        av = np.ascontiguousarray(np.asarray(edgelet_angles, dtype=np.float64))
        cfg.dict_kind = OSAR_DICT_EDGELET
        cfg.n_atoms = 0
        cfg.n_edgelet_lengths, cfg.edgelet_lengths = int(lv.size), lv.ctypes.data
        cfg.n_edgelet_angles, cfg.edgelet_angles_deg = int(av.size), av.ctypes.data
        keep = (lv, av)
    else:
        d = np.asarray(dictionary, dtype=np.complex128)
        keep = np.asfortranarray(d)
        cfg.dict_kind = OSAR_DICT_HOST
        cfg.n_atoms = d.shape[1]
        cfg.dict_c128 = keep.ctypes.data
    cfg.lam = float(lam)
    cfg.lambda_relative = 1 if lambda_relative else 0
    cfg.power_iters_first = int(power_iters_first)
    cfg.power_iters = int(power_iters)
    cfg.lipschitz_margin = float(lipschitz_margin)
    cfg.restart_momentum = 1 if restart_momentum else 0
    cfg.compensated = 1 if compensated else 0
    cfg.cuda_stream = stream
    cfg.overlap_synthesis = 1 if overlap_synthesis else 0
    cfg.synth_ctas = int(synth_ctas)
    cfg.tc_pairs = int(tc_pairs)  # bit 0 dictionary product, bit 1 Gram update
    cfg.fuse_first_step = 1 if fuse_first_step else 0
    cfg.defer_gram = 1 if defer_gram else 0
    cfg.guard_bytes = int(guard_bytes)
    cfg.fuse_power_gram = 1 if fuse_power_gram else 0
    cfg.pixel_gram = 1 if pixel_gram else 0
    cfg.gram_superblock = int(gram_superblock)
    cfg.gram_ahead = int(gram_ahead)
    if lambdas is not None and len(lambdas) > 1:
        # lambda path: one solution per value (relative or absolute like lam)
        lv = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
        cfg.n_lambdas = int(lv.size)
        cfg.lambda_list = lv.ctypes.data
        keep = (keep, lv)
    elif lambdas is not None:
        cfg.lam = float(lambdas[0])
    cfg._keepalive = keep
    return cfg


class Osar:
    """One online reconstruction context (owns its device memory)."""

    def __init__(self, cfg: Optional[OsarConfig] = None, _handle=None, **kw):
        self._lib = load_library()
        self._h = None
        if _handle is not None:
            self._h = _handle
            self.cfg = cfg
        else:
            self.cfg = cfg if cfg is not None else make_config(**kw)
            h = C.c_void_p()
            st = self._lib.osar_create(C.byref(self.cfg), C.byref(h))
            if st != OSAR_OK:
                raise OsarError(st, self._lib.osar_last_error(None).decode())
            self._h = h
        m, n, k = C.c_int32(), C.c_int32(), C.c_int32()
        self._lib.osar_get_dims(self._h, C.byref(m), C.byref(n), C.byref(k))
        self.m_atoms, self.n_pixels, self.n_freq = m.value, n.value, k.value
        # the stored Gram's order: M, or N in the pixel-space Gram form
        pixel = self.cfg is not None and getattr(self.cfg, "pixel_gram", 0)
        self.gram_dim = self.n_pixels if pixel else self.m_atoms

    # -- helpers --------------------------------------------------------
    def _check(self, st: int):
        if st != OSAR_OK:
            raise OsarError(st, self._lib.osar_last_error(self._h).decode())

    def close(self):
        if self._h is not None:
            self._lib.osar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- Eqs. 12-13 and Algorithm 1 ---------------------------------------
    def push_pulse(self, gamma, d, noise_var=None):
        """One pulse; noise_var: its n_freq noise variances (R_n diagonal),
        None for white noise."""
        g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
        dv = _c128(d)
        if dv.size != self.n_freq or g.size != 3:
            raise ValueError("gamma must have 3 entries and d n_freq entries")
        if noise_var is None:
            self._check(self._lib.osar_push_pulse(self._h, _dptr(g),
                                                  _dptr(dv.view(np.float64))))
            return
        vv = np.ascontiguousarray(np.asarray(noise_var, dtype=np.float64))
        if vv.size != self.n_freq:
            raise ValueError("noise_var needs n_freq entries")
        self._check(self._lib.osar_push_pulse_var(self._h, _dptr(g),
                                                  _dptr(dv.view(np.float64)), _dptr(vv)))

    def push_pulse_dev(self, gamma, d_dev_ptr: int):
        g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
        self._check(self._lib.osar_push_pulse_dev(self._h, _dptr(g), C.c_void_p(d_dev_ptr)))

    def iterate(self, max_iters: int, tol: float = 0.0, want_count: bool = True):
        cnt = C.c_int32(0)
        self._check(self._lib.osar_iterate(
            self._h, int(max_iters), float(tol), C.byref(cnt) if want_count else None))
        return cnt.value if want_count else None

    def coeffs(self) -> np.ndarray:
        out = np.empty(self.m_atoms, dtype=np.complex128)
        self._check(self._lib.osar_get_coeffs(self._h, _dptr(out.view(np.float64))))
        return out

    def coeffs_dev(self, out_ptr: int):
        self._check(self._lib.osar_get_coeffs_dev(self._h, C.c_void_p(out_ptr)))

    def coeffs_async(self, out: np.ndarray, slot: int = 0):
        """Queue a copy of c_hat into `out` (complex128, M entries, ideally
        pinned); it is valid after wait_coeffs(slot)."""
        if out.dtype != np.complex128 or out.size < self.m_atoms or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous complex128 array of M entries")
        self._check(self._lib.osar_get_coeffs_async(self._h, _dptr(out.view(np.float64)),
                                                    int(slot)))

    def wait_coeffs(self, slot: int = 0):
        self._check(self._lib.osar_wait_coeffs(self._h, int(slot)))

    def state(self) -> dict:
        n = C.c_int32()
        lip, lam, t = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.osar_get_state(self._h, C.byref(n), C.byref(lip),
                                             C.byref(lam), C.byref(t)))
        return {"n": n.value, "lipschitz": lip.value, "lambda": lam.value, "t": t.value}

    def lambda_state(self, l: int) -> dict:
        """Solution l of a lambda path: coefficients, lambda_n, t and the FISTA
        steps of the last iterate call."""
        out = np.empty(self.m_atoms, dtype=np.complex128)
        lam, t = C.c_double(), C.c_double()
        it = C.c_int32()
        self._check(self._lib.osar_get_lambda_state(
            self._h, int(l), _dptr(out.view(np.float64)), C.byref(lam), C.byref(t),
            C.byref(it)))
        return {"coeffs": out, "lambda": lam.value, "t": t.value, "iters": it.value}

    def gram(self) -> np.ndarray:
        out = np.empty((self.gram_dim, self.gram_dim), dtype=np.complex128)
        self._check(self._lib.osar_get_gram(self._h, _dptr(out.view(np.float64))))
        return out

    def gram_entries(self, rows, cols) -> np.ndarray:
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
        c = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
        out = np.empty(r.size, dtype=np.complex128)
        self._check(self._lib.osar_get_gram_entries(
            self._h, r.ctypes.data_as(C.POINTER(C.c_int32)),
            c.ctypes.data_as(C.POINTER(C.c_int32)), int(r.size),
            _dptr(out.view(np.float64))))
        return out

    def b(self) -> np.ndarray:
        out = np.empty(self.m_atoms, dtype=np.complex128)
        self._check(self._lib.osar_get_b(self._h, _dptr(out.view(np.float64))))
        return out

    def gram_apply(self, x) -> np.ndarray:
        xv = _c128(x)
        out = np.empty(self.gram_dim, dtype=np.complex128)
        self._check(self._lib.osar_gram_apply(self._h, _dptr(xv.view(np.float64)),
                                              _dptr(out.view(np.float64))))
        return out

    def gram_apply_static(self, x_dev_ptr: int, y_dev_ptr: int):
        """y = A x on caller device buffers with no allocation (asynchronous
        on the context's stream; see osar_gram_apply_static)."""
        self._check(self._lib.osar_gram_apply_static(
            self._h, C.c_void_p(x_dev_ptr), C.c_void_p(y_dev_ptr)))

    def metrics(self, threshold: float = 2e-2, support=None) -> dict:
        """Large-coefficient count and the coefficient-domain SNR of c_hat
        against a reference support (osar_get_metrics)."""
        out = OsarMetrics()
        if support is None:
            sp, n = None, 0
        else:
            sv = np.ascontiguousarray(np.asarray(support, dtype=np.int32))
            sp, n = sv.ctypes.data_as(C.POINTER(C.c_int32)), int(sv.size)
        self._check(self._lib.osar_get_metrics(self._h, float(threshold), sp, n,
                                               C.byref(out)))
        return {k: getattr(out, k) for k, _ in OsarMetrics._fields_}

    def simulate_pulse(self, gamma, coeffs) -> np.ndarray:
        g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
        cv = _c128(coeffs)
        out = np.empty(self.n_freq, dtype=np.complex128)
        self._check(self._lib.osar_simulate_pulse(self._h, _dptr(g), _dptr(cv.view(np.float64)),
                                                  _dptr(out.view(np.float64))))
        return out

    def unroll_grad(self, steps: int, ckpt_every: int, lam: float, tau: float,
                    c0, c_true, t0: float = 1.0) -> dict:
        """Loss ||c_T - c_true||^2 after `steps` unrolled inner steps on the
        current Gram and data vector, and its gradients with respect to
        lambda, tau and b (adjoint kernels, checkpoints every ckpt_every)."""
        c0v = _c128(c0)
        ctv = _c128(c_true)
        loss, dl, dt = C.c_double(), C.c_double(), C.c_double()
        db = np.empty(self.m_atoms, dtype=np.complex128)
        ct = np.empty(self.m_atoms, dtype=np.complex128)
        self._check(self._lib.osar_unroll_grad(
            self._h, int(steps), int(ckpt_every), float(lam), float(tau),
            float(t0), _dptr(c0v.view(np.float64)), _dptr(ctv.view(np.float64)),
            C.byref(loss), C.byref(dl), C.byref(dt), _dptr(db.view(np.float64)),
            _dptr(ct.view(np.float64))))
        return {"loss": loss.value, "d_lambda": dl.value, "d_tau": dt.value,
                "d_b": db, "c_T": ct}

    def set_lambda(self, lam: float, l: int = 0):
        """Lambda setting of solution l from the next pulse on (a factor of
        ||b_n||_inf when the context is relative)."""
        self._check(self._lib.osar_set_lambda(self._h, int(l), float(lam)))

    def set_gram_ahead(self, mode: int):
        """The Gram update's schedule from the next push on (0, 1 or 2)."""
        self._check(self._lib.osar_set_gram_ahead(self._h, int(mode)))

    def data_grad(self, gamma, d_b) -> np.ndarray:
        """dL/dd_s = G_s dL/db for the pulse at gamma (the forward model
        applied to the b-gradient)."""
        return self.simulate_pulse(gamma, d_b)

    def synchronize(self):
        self._check(self._lib.osar_synchronize(self._h))

    def last_error(self) -> str:
        return self._lib.osar_last_error(self._h).decode()

    def check_guards(self) -> int:
        """Number of device buffers whose guard region was overwritten."""
        n = C.c_int32(0)
        self._check(self._lib.osar_check_guards(self._h, C.byref(n)))
        return int(n.value)

    def poke_guard(self, index: int) -> int:
        return int(self._lib.osar_poke_guard(self._h, int(index)))

    def probe_bounded_wait(self, limit_ns: int) -> int:
        """Run the failure-detection check (a bounded wait that nothing
        completes); returns the status, OSAR_E_TIMEOUT when it gave up as
        designed."""
        return int(self._lib.osar_probe_bounded_wait(self._h, int(limit_ns)))

    # -- profiling ----------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._check(self._lib.osar_profile_enable(self._h, 1 if on else 0))

    def profile_reset(self):
        self._check(self._lib.osar_profile_reset(self._h))

    def profile_passes(self) -> int:
        n = C.c_int64()
        self._check(self._lib.osar_profile_passes(self._h, C.byref(n)))
        return n.value

    def profile_select(self, *kernels: str):
        """Bracket only these kernel classes (names of KERNEL_CLASSES) while
        profiling is on; no names selects every class."""
        mask = 0
        for k in kernels:
            mask |= 1 << KERNEL_CLASSES[k]
        self._check(self._lib.osar_profile_select(
            self._h, mask if kernels else (1 << len(KERNEL_CLASSES)) - 1))

    def profile_ahead(self, with_grid: bool = False):
        """Pushes since the last profile reset whose Gram update ran ahead
        (and, with_grid, the side stream's SMs of the last one)."""
        n, g = C.c_int64(), C.c_int32()
        self._check(self._lib.osar_profile_ahead(self._h, C.byref(n), C.byref(g)))
        return (n.value, g.value) if with_grid else n.value

    def profile_sample(self, kernel: str, every: int):
        """Bracket one launch in `every` of this class."""
        self._check(self._lib.osar_profile_sample(self._h, KERNEL_CLASSES[kernel], every))

    def profile_read(self, kernel: str):
        n = C.c_int64()
        ms = C.c_double()
        self._check(self._lib.osar_profile_read(self._h, KERNEL_CLASSES[kernel],
                                                C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self._lib.osar_launch_count(self._h, C.byref(n)))
        return n.value

    def device_bytes(self) -> int:
        n = C.c_int64()
        self._check(self._lib.osar_device_bytes(self._h, C.byref(n)))
        return n.value

    # -- checkpoints ----------------------------------------------------------
    def save(self, path: str):
        self._check(self._lib.osar_save(self._h, path.encode()))

    @classmethod
    def load(cls, path: str, cfg: OsarConfig) -> "Osar":
        lib = load_library()
        h = C.c_void_p()
        st = lib.osar_load(path.encode(), C.byref(cfg), C.byref(h))
        if st != OSAR_OK:
            raise OsarError(st, lib.osar_last_error(None).decode())
        return cls(cfg, _handle=h)


class OsarBatch:
    """Many independent online reconstructions of uneven size (batching
    form); scene s behaves like its own Osar context."""

    def __init__(self, cfgs, stream=None):
        self._lib = load_library()
        self._h = None
        self.cfgs = list(cfgs)
        arr = (OsarConfig * len(self.cfgs))(*self.cfgs)
        h = C.c_void_p()
        st = self._lib.osar_batch_create(arr, len(self.cfgs),
                                         C.c_void_p(stream) if stream else None,
                                         C.byref(h))
        if st != OSAR_OK:
            raise OsarError(st, self._lib.osar_batch_last_error(None).decode())
        self._h = h
        self.n_scenes = len(self.cfgs)
        self.m_atoms = [c.nx * c.ny for c in self.cfgs]
        self.n_freq = [c.n_freq for c in self.cfgs]
        self.stride = max(self.n_freq)

    def _check(self, st):
        if st != OSAR_OK:
            raise OsarError(st, self._lib.osar_batch_last_error(self._h).decode())

    def close(self):
        if self._h is not None:
            self._lib.osar_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, active, gammas, data):
        """active: n_scenes flags; gammas: n_scenes x 3; data: list of the
        active scenes' pulse samples (entries of inactive scenes ignored)."""
        S = self.n_scenes
        act = np.ascontiguousarray(np.asarray(active, dtype=np.int32))
        gam = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).reshape(S, 3))
        d = np.zeros((S, self.stride), dtype=np.complex128)
        for s in range(S):
            if act[s]:
                d[s, :self.n_freq[s]] = data[s]
        self._check(self._lib.osar_batch_push(
            self._h, act.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(gam),
            _dptr(d.view(np.float64)), self.stride))

    def iterate(self, max_iters, tol=0.0, want_counts=True):
        cnt = np.zeros(self.n_scenes, dtype=np.int32)
        self._check(self._lib.osar_batch_iterate(
            self._h, int(max_iters), float(tol),
            cnt.ctypes.data_as(C.POINTER(C.c_int32)) if want_counts else None))
        return cnt if want_counts else None

    def coeffs(self, scene):
        out = np.empty(self.m_atoms[scene], dtype=np.complex128)
        self._check(self._lib.osar_batch_get_coeffs(self._h, int(scene),
                                                    _dptr(out.view(np.float64))))
        return out

    def state(self, scene):
        n = C.c_int32()
        lip, lam, t = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.osar_batch_get_state(self._h, int(scene), C.byref(n),
                                                   C.byref(lip), C.byref(lam), C.byref(t)))
        return {"n": n.value, "lipschitz": lip.value, "lambda": lam.value, "t": t.value}

    def autotune(self):
        ch = C.c_int32()
        self._check(self._lib.osar_batch_autotune(self._h, C.byref(ch)))
        return ch.value

    def tuning(self) -> dict:
        seg, sb, lpt = C.c_int32(), C.c_int32(), C.c_int32()
        d0, d1 = C.c_double(), C.c_double()
        self._check(self._lib.osar_batch_get_tuning(self._h, C.byref(seg), C.byref(sb),
                                                    C.byref(lpt), C.byref(d0),
                                                    C.byref(d1)))
        return {"segment_blocks": seg.value, "gram_superblock": sb.value,
                "gram_largest_first": bool(lpt.value), "gram_ms_default": d0.value,
                "gram_ms_chosen": d1.value}

    def info(self):
        n, seg = C.c_int32(), C.c_int32()
        b, l = C.c_int64(), C.c_int64()
        self._check(self._lib.osar_batch_info(self._h, C.byref(n), C.byref(b),
                                              C.byref(l), C.byref(seg)))
        return {"n_scenes": n.value, "device_bytes": b.value, "launches": l.value,
                "segment_blocks": seg.value}

    def synchronize(self):
        self._check(self._lib.osar_batch_synchronize(self._h))

    def check_guards(self) -> int:
        n = C.c_int32(0)
        self._check(self._lib.osar_batch_check_guards(self._h, C.byref(n)))
        return int(n.value)


def version() -> str:
    return load_library().osar_version().decode()
