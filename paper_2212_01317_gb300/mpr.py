"""Thin ctypes binding of libmpr (include/mpr.h), same names as the C-ABI.

Argument marshalling only: every step of the method runs in the CUDA library.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); device
tensors are passed as device pointers. The library must be built for sm_103a
(``paper_2212_01317_gb300.build``); without it, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MPR_OK, MPR_EINVAL, MPR_ENOMEM, MPR_ECUDA, MPR_ENOSAMPLES, MPR_ETIMEOUT, MPR_ESTATE = range(7)
MPR_STORE_F32, MPR_STORE_BF16, MPR_STORE_F16 = 0, 1, 2
MPR_INIT_BLOCK_MEAN, MPR_INIT_RANDOM = 0, 1
MPR_STOP_CROSS, MPR_STOP_WINDOW = 0, 1
MPR_CURVE_POINTS = 40

EXPORTS = [
    "mpr_default_options", "mpr_create", "mpr_destroy", "mpr_last_error", "mpr_status_string",
    "mpr_get_info", "mpr_calibrate", "mpr_set_temperatures", "mpr_get_temperatures",
    "mpr_simulate", "mpr_predict", "mpr_get_block_stats", "mpr_sim_begin", "mpr_sim_sweep",
    "mpr_sim_end", "mpr_halfstep", "mpr_get_state", "mpr_set_state", "mpr_get_stop",
    "mpr_set_running", "mpr_block_energy", "mpr_get_block_e", "mpr_get_profile",
    "mpr_block_stats_noalloc", "mpr_set_realization_base", "mpr_get_accumulator",
    "mpr_set_accumulator", "mpr_smooth_temperatures", "mpr_set_site_temperatures",
    "mpr_get_site_temperatures", "mpr_energy_moments", "mpr_energy_vjp", "mpr_create_batch",
    "mpr_get_energy_curve", "mpr_set_energy_curve", "mpr_sample_chains",
    "mpr_predict_batch", "mpr_get_slice_layout", "mpr_autotune", "mpr_release_cached_memory",
    "mpr3_create", "mpr3_destroy", "mpr3_last_error", "mpr3_get_info", "mpr3_get_block_stats",
    "mpr3_calibrate", "mpr3_set_temperatures", "mpr3_simulate", "mpr3_predict", "mpr3_sim_begin",
    "mpr3_halfstep", "mpr3_get_state", "mpr3_set_state", "mpr3_sim_end", "mpr3_get_profile",
]
MPR_NOALLOC_MAX_BLOCKS = 65536


class mpr_grid(C.Structure):
    _fields_ = [("height", C.c_int32), ("width", C.c_int32), ("block", C.c_int32)]


class mpr_options(C.Structure):
    _fields_ = [("q", C.c_double), ("J", C.c_double), ("seed", C.c_uint64),
                ("slice_id", C.c_uint32), ("n_max", C.c_int32), ("n_eq", C.c_int32),
                ("n_meas", C.c_int32), ("n_bisect", C.c_int32), ("cal_chains", C.c_int32),
                ("t_lo", C.c_float), ("t_hi", C.c_float), ("overrelax", C.c_int32),
                ("init", C.c_int32), ("storage", C.c_int32), ("group", C.c_int32),
                ("profile", C.c_int32), ("cal_mode", C.c_int32), ("wait_ms", C.c_int32),
                ("barrier_test", C.c_int32), ("cal_method", C.c_int32), ("n_newton", C.c_int32),
                ("t_init", C.c_float), ("sim_graph", C.c_int32), ("cal_points", C.c_int32),
                ("sim_tail", C.c_int32), ("sweep_form", C.c_int32), ("pair_tail", C.c_int32),
                ("sweep_form_bulk", C.c_int32), ("stop_rule", C.c_int32), ("n_fit", C.c_int32),
                ("n_f", C.c_int32), ("cal_warm", C.c_float), ("alloc_test", C.c_int32),
                ("cal_continue", C.c_int32), ("cal_sweep", C.c_int32),
                ("cuda_stream", C.c_void_p)]


class mpr_profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("sim_halfstep_launches", C.c_int64),
                ("cal_halfstep_launches", C.c_int64), ("sim_halfstep_ms", C.c_double),
                ("cal_halfstep_ms", C.c_double), ("sim_tail_launches", C.c_int64),
                ("sim_tail_updates", C.c_int64), ("sim_tail_ms", C.c_double)]


class mpr_grid3(C.Structure):
    _fields_ = [("depth", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("block", C.c_int32)]


class mpr3_info(C.Structure):
    _fields_ = [("depth", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("block", C.c_int32), ("nblk", C.c_int32), ("n_gap", C.c_int64),
                ("zmin", C.c_double), ("zmax", C.c_double), ("realizations", C.c_int64),
                ("gap_updates", C.c_int64), ("cal_gap_updates", C.c_int64)]


class mpr_tuning(C.Structure):
    _fields_ = [("group", C.c_int32), ("form", C.c_int32), ("ms", C.c_float * 4),
                ("trial_ms", C.c_float)]


class mpr_info(C.Structure):
    _fields_ = [("height", C.c_int32), ("width", C.c_int32), ("block", C.c_int32),
                ("nbx", C.c_int32), ("nby", C.c_int32), ("nblk", C.c_int32),
                ("n_gap", C.c_int64), ("n_gap_colour", C.c_int64 * 2),
                ("zmin", C.c_double), ("zmax", C.c_double), ("degenerate", C.c_int32),
                ("calibrated", C.c_int32), ("realizations", C.c_int64), ("batch", C.c_int32),
                ("group", C.c_int32), ("gap_updates", C.c_int64),
                ("cal_gap_updates", C.c_int64), ("device_bytes", C.c_int64),
                ("n_slices", C.c_int32)]


class MprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_STATUS_NAMES = {0: "MPR_OK", 1: "MPR_EINVAL", 2: "MPR_ENOMEM", 3: "MPR_ECUDA",
                 4: "MPR_ENOSAMPLES", 5: "MPR_ETIMEOUT", 6: "MPR_ESTATE"}

_lib = None


def load(path: str | None = None):
    """Loads libmpr.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if not _build.up_to_date():
            _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libmpr.so not found at {path}; build it with "
                          "paper_2212_01317_gb300.build.build()")
    L = C.CDLL(path)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    st = C.c_int
    sig = {
        "mpr_default_options": (None, [C.POINTER(mpr_options)]),
        "mpr_create": (st, [C.POINTER(mpr_grid), P, P, C.POINTER(mpr_options), C.POINTER(P)]),
        "mpr_destroy": (None, [P]),
        "mpr_release_cached_memory": (None, []),
        "mpr_last_error": (C.c_char_p, [P]),
        "mpr_status_string": (C.c_char_p, [st]),
        "mpr_get_info": (st, [P, C.POINTER(mpr_info)]),
        "mpr_calibrate": (st, [P, P]),
        "mpr_set_temperatures": (st, [P, P]),
        "mpr_get_temperatures": (st, [P, P]),
        "mpr_simulate": (st, [P, i32]),
        "mpr_predict": (st, [P, P, P, P]),
        "mpr_get_block_stats": (st, [P, P, P, P, P, P]),
        "mpr_sim_begin": (st, [P, i32]),
        "mpr_sim_sweep": (st, [P, i32, C.POINTER(i64)]),
        "mpr_sim_end": (st, [P]),
        "mpr_halfstep": (st, [P, i32, i32, i32]),
        "mpr_get_state": (st, [P, i32, P]),
        "mpr_set_state": (st, [P, i32, P]),
        "mpr_get_stop": (st, [P, P, P]),
        "mpr_set_running": (st, [P, P]),
        "mpr_block_energy": (st, [P, i32, P]),
        "mpr_get_block_e": (st, [P, P]),
        "mpr_get_profile": (st, [P, C.POINTER(mpr_profile)]),
        "mpr_block_stats_noalloc": (st, [C.POINTER(mpr_grid), P, P, C.c_double, C.c_double, P, P,
                                         P, P, P, P, P]),
        "mpr_set_realization_base": (st, [P, i64]),
        "mpr_get_accumulator": (st, [P, P, C.POINTER(i64)]),
        "mpr_set_accumulator": (st, [P, P, i64]),
        "mpr_smooth_temperatures": (st, [P, i32, i32, P]),
        "mpr_set_site_temperatures": (st, [P, P]),
        "mpr_get_site_temperatures": (st, [P, P]),
        "mpr_energy_moments": (st, [P, P, i32, i32, i32, i32, P, P, P, P]),
        "mpr_energy_vjp": (st, [P, P, P]),
        "mpr_create_batch": (st, [i32, P, P, P, C.POINTER(mpr_options), C.POINTER(P)]),
        "mpr_predict_batch": (st, [P, P, P, P]),
        "mpr_get_slice_layout": (st, [P, P]),
        "mpr_autotune": (st, [P, i32, i32, C.POINTER(mpr_tuning)]),
        "mpr_get_energy_curve": (st, [P, P, P, i32, C.POINTER(i32)]),
        "mpr_set_energy_curve": (st, [P, P, P, i32]),
        "mpr_sample_chains": (st, [P, i32, i32, i32]),
        "mpr3_create": (st, [C.POINTER(mpr_grid3), P, P, C.POINTER(mpr_options), C.POINTER(P)]),
        "mpr3_destroy": (None, [P]),
        "mpr3_last_error": (C.c_char_p, [P]),
        "mpr3_get_info": (st, [P, C.POINTER(mpr3_info)]),
        "mpr3_get_block_stats": (st, [P, P, P, P, P, P]),
        "mpr3_calibrate": (st, [P, P]),
        "mpr3_set_temperatures": (st, [P, P]),
        "mpr3_simulate": (st, [P, i32]),
        "mpr3_predict": (st, [P, P, P, P]),
        "mpr3_get_profile": (st, [P, C.POINTER(mpr_profile)]),
        "mpr3_sim_begin": (st, [P, i32]),
        "mpr3_halfstep": (st, [P, i32, i32, i32]),
        "mpr3_get_state": (st, [P, i32, P]),
        "mpr3_set_state": (st, [P, i32, P]),
        "mpr3_sim_end": (st, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "arrays must be C-contiguous"
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, status: int):
    if status != MPR_OK:
        msg = load().mpr_last_error(ctx).decode() if ctx else ""
        raise MprError(status, msg or load().mpr_status_string(status).decode())


def mpr_default_options(**kw) -> mpr_options:
    o = mpr_options()
    load().mpr_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def mpr_create(height: int, width: int, block: int, mask, values, options: mpr_options | None = None):
    g = mpr_grid(height, width, block)
    out = C.c_void_p()
    st = load().mpr_create(C.byref(g), _ptr(mask), _ptr(values),
                           None if options is None else C.byref(options), C.byref(out))
    if st != MPR_OK:
        raise MprError(st, load().mpr_status_string(st).decode())
    return out


def mpr_create_batch(grids, masks, values, options: mpr_options | None = None):
    """grids: list of (height, width, block); masks / values: lists of arrays or
    tensors (host or device), one per field."""
    n = len(grids)
    g = (mpr_grid * n)(*[mpr_grid(h, w, b) for (h, w, b) in grids])
    mp = (C.c_void_p * n)(*[_ptr(m).value for m in masks])
    vp = (C.c_void_p * n)(*[_ptr(v).value for v in values])
    out = C.c_void_p()
    st = load().mpr_create_batch(n, g, mp, vp, None if options is None else C.byref(options),
                                 C.byref(out))
    if st != MPR_OK:
        raise MprError(st, load().mpr_status_string(st).decode())
    return out


def mpr_predict_batch(ctx, outs, truths=None, aae_rase=None):
    n = len(outs)
    op = (C.c_void_p * n)(*[_ptr(o).value for o in outs])
    tp = None if truths is None else (C.c_void_p * n)(*[_ptr(t).value for t in truths])
    _check(ctx, load().mpr_predict_batch(ctx, op, tp, _ptr(aae_rase)))


def mpr_get_slice_layout(ctx, n: int) -> np.ndarray:
    r = np.zeros((n, 4), np.int32)
    _check(ctx, load().mpr_get_slice_layout(ctx, _ptr(r)))
    return r


def mpr_autotune(ctx, n_realizations: int, n_sweeps: int = 4) -> mpr_tuning:
    t = mpr_tuning()
    _check(ctx, load().mpr_autotune(ctx, int(n_realizations), int(n_sweeps), C.byref(t)))
    return t


def mpr_destroy(ctx):
    load().mpr_destroy(ctx)


def mpr_release_cached_memory():
    """Returns the library's cached (unused) device memory to the device."""
    load().mpr_release_cached_memory()


def mpr_get_info(ctx) -> mpr_info:
    info = mpr_info()
    _check(ctx, load().mpr_get_info(ctx, C.byref(info)))
    return info


def mpr_calibrate(ctx, block_T_out=None):
    _check(ctx, load().mpr_calibrate(ctx, _ptr(block_T_out)))


def mpr_get_energy_curve(ctx, capacity: int = 64):
    """The context's unconditional e(T) curve (measured on first use):
    (T float32[n], e float64[n])."""
    T = np.zeros(capacity, np.float32)
    e = np.zeros(capacity, np.float64)
    n = C.c_int32()
    _check(ctx, load().mpr_get_energy_curve(ctx, _ptr(T), _ptr(e), capacity, C.byref(n)))
    return T[:n.value].copy(), e[:n.value].copy()


def mpr_set_energy_curve(ctx, T, e):
    T = np.ascontiguousarray(T, dtype=np.float32)
    e = np.ascontiguousarray(e, dtype=np.float64)
    _check(ctx, load().mpr_set_energy_curve(ctx, _ptr(T), _ptr(e), int(T.size)))


def mpr_sample_chains(ctx, n_chains: int, n_equil: int, n_samples: int):
    _check(ctx, load().mpr_sample_chains(ctx, int(n_chains), int(n_equil), int(n_samples)))


def mpr_set_temperatures(ctx, T):
    _check(ctx, load().mpr_set_temperatures(ctx, _ptr(T)))


def mpr_get_temperatures(ctx, out):
    _check(ctx, load().mpr_get_temperatures(ctx, _ptr(out)))


def mpr_simulate(ctx, n_realizations: int):
    _check(ctx, load().mpr_simulate(ctx, int(n_realizations)))


def mpr_predict(ctx, out, truth=None, aae_rase=None):
    _check(ctx, load().mpr_predict(ctx, _ptr(out), _ptr(truth), _ptr(aae_rase)))


def mpr_get_block_stats(ctx, Es=None, Nsp=None, Nb=None, mean_angle=None, n_gap=None):
    _check(ctx, load().mpr_get_block_stats(ctx, _ptr(Es), _ptr(Nsp), _ptr(Nb), _ptr(mean_angle),
                                           _ptr(n_gap)))


def mpr_sim_begin(ctx, n_realizations: int):
    _check(ctx, load().mpr_sim_begin(ctx, int(n_realizations)))


def mpr_sim_sweep(ctx, n_sweeps: int) -> int:
    left = C.c_int64()
    _check(ctx, load().mpr_sim_sweep(ctx, int(n_sweeps), C.byref(left)))
    return left.value


def mpr_sim_end(ctx):
    _check(ctx, load().mpr_sim_end(ctx))


def mpr_halfstep(ctx, colour: int, t: int, tag: int = 0):
    _check(ctx, load().mpr_halfstep(ctx, colour, t, tag))


def mpr_get_state(ctx, r: int, out):
    _check(ctx, load().mpr_get_state(ctx, r, _ptr(out)))


def mpr_set_state(ctx, r: int, angles):
    _check(ctx, load().mpr_set_state(ctx, r, _ptr(angles)))


def mpr_get_stop(ctx, stop_sweep=None, running=None):
    _check(ctx, load().mpr_get_stop(ctx, _ptr(stop_sweep), _ptr(running)))


def mpr_set_running(ctx, running):
    _check(ctx, load().mpr_set_running(ctx, _ptr(running)))


def mpr_block_energy(ctx, r: int, out):
    _check(ctx, load().mpr_block_energy(ctx, r, _ptr(out)))


def mpr_get_profile(ctx) -> mpr_profile:
    p = mpr_profile()
    _check(ctx, load().mpr_get_profile(ctx, C.byref(p)))
    return p


def mpr_get_block_e(ctx, out):
    _check(ctx, load().mpr_get_block_e(ctx, _ptr(out)))


def mpr_smooth_temperatures(ctx, r_s: int, n_s: int, T_site_out=None):
    _check(ctx, load().mpr_smooth_temperatures(ctx, int(r_s), int(n_s), _ptr(T_site_out)))


def mpr_set_site_temperatures(ctx, T_site=None):
    _check(ctx, load().mpr_set_site_temperatures(ctx, _ptr(T_site)))


def mpr_get_site_temperatures(ctx, out):
    _check(ctx, load().mpr_get_site_temperatures(ctx, _ptr(out)))


def mpr_energy_moments(ctx, beta, n_eq: int, n_meas: int, tag: int, restart: bool,
                       mean_e=None, var_E=None, cov_r=None, cov_d=None):
    _check(ctx, load().mpr_energy_moments(ctx, _ptr(beta), int(n_eq), int(n_meas), int(tag),
                                          1 if restart else 0, _ptr(mean_e), _ptr(var_E),
                                          _ptr(cov_r), _ptr(cov_d)))


def mpr_energy_vjp(ctx, grad_e, grad_beta):
    _check(ctx, load().mpr_energy_vjp(ctx, _ptr(grad_e), _ptr(grad_beta)))


def mpr_set_realization_base(ctx, r_first: int):
    _check(ctx, load().mpr_set_realization_base(ctx, int(r_first)))


def mpr_get_accumulator(ctx, sum_out=None) -> int:
    n = C.c_int64()
    _check(ctx, load().mpr_get_accumulator(ctx, _ptr(sum_out), C.byref(n)))
    return n.value


def mpr_set_accumulator(ctx, sum_in, n_realizations: int):
    _check(ctx, load().mpr_set_accumulator(ctx, _ptr(sum_in), int(n_realizations)))


def mpr_block_stats_noalloc(height: int, width: int, block: int, mask, values, Es, Nsp, Nb,
                            mean_angle, n_gap, zrange, q: float = 0.5, J: float = 1.0,
                            cuda_stream=None) -> int:
    """Block statistics without allocation; every array a CUDA tensor. Returns the status."""
    g = mpr_grid(height, width, block)
    return load().mpr_block_stats_noalloc(C.byref(g), _ptr(mask), _ptr(values), q, J, _ptr(Es),
                                          _ptr(Nsp), _ptr(Nb), _ptr(mean_angle), _ptr(n_gap),
                                          _ptr(zrange), cuda_stream)


class GapFiller:
    """Owns one mpr context; numpy in, numpy out (marshalling only)."""

    def __init__(self, values, mask, block: int, **options):
        values = np.ascontiguousarray(values, dtype=np.float32)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.H, self.W = mask.shape
        self.opt = mpr_default_options(**options)
        self.ctx = mpr_create(self.H, self.W, block, mask, values, self.opt)
        self.info = mpr_get_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            mpr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nblk(self) -> int:
        return self.info.nblk

    def refresh(self) -> mpr_info:
        self.info = mpr_get_info(self.ctx)
        return self.info

    def calibrate(self) -> np.ndarray:
        T = np.zeros(self.nblk, np.float32)
        mpr_calibrate(self.ctx, T)
        return T

    def set_temperatures(self, T):
        mpr_set_temperatures(self.ctx, np.ascontiguousarray(T, dtype=np.float32))

    def energy_curve(self):
        return mpr_get_energy_curve(self.ctx)

    def sample_chains(self, n_chains: int, n_equil: int, n_samples: int):
        mpr_sample_chains(self.ctx, n_chains, n_equil, n_samples)

    def set_energy_curve(self, T, e):
        mpr_set_energy_curve(self.ctx, T, e)

    def simulate(self, n: int):
        mpr_simulate(self.ctx, n)

    def predict(self, truth=None):
        out = np.zeros((self.H, self.W), np.float32)
        if truth is None:
            mpr_predict(self.ctx, out)
            return out, None
        err = np.zeros(2, np.float64)
        mpr_predict(self.ctx, out, np.ascontiguousarray(truth, dtype=np.float32), err)
        return out, (float(err[0]), float(err[1]))

    def block_stats(self):
        n = self.nblk
        Es, Nsp, Nb = np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32)
        ma, ng = np.zeros(n, np.float32), np.zeros(n, np.int32)
        mpr_get_block_stats(self.ctx, Es, Nsp, Nb, ma, ng)
        return Es, Nsp, Nb, ma, ng

    def smooth_temperatures(self, r_s: int, n_s: int) -> np.ndarray:
        out = np.zeros((self.H, self.W), np.float32)
        mpr_smooth_temperatures(self.ctx, r_s, n_s, out)
        return out

    def set_site_temperatures(self, T_site):
        mpr_set_site_temperatures(
            self.ctx, None if T_site is None else np.ascontiguousarray(T_site, dtype=np.float32))

    # step-wise access
    def sim_begin(self, n: int):
        mpr_sim_begin(self.ctx, n)

    def sim_sweep(self, n: int = 1) -> int:
        return mpr_sim_sweep(self.ctx, n)

    def sim_end(self):
        mpr_sim_end(self.ctx)

    def halfstep(self, colour: int, t: int, tag: int = 0):
        mpr_halfstep(self.ctx, colour, t, tag)

    def get_state(self, r: int) -> np.ndarray:
        out = np.zeros((self.H, self.W), np.float32)
        mpr_get_state(self.ctx, r, out)
        return out

    def set_state(self, r: int, angles):
        mpr_set_state(self.ctx, r, np.ascontiguousarray(angles, dtype=np.float32))

    def get_stop(self, R: int):
        stop = np.zeros((R, self.nblk), np.int32)
        run = np.zeros((R, self.nblk), np.uint8)
        mpr_get_stop(self.ctx, stop, run)
        return stop, run

    def set_running(self, running):
        mpr_set_running(self.ctx, np.ascontiguousarray(running, dtype=np.uint8))

    def block_e(self, R: int) -> np.ndarray:
        e = np.zeros((R, self.nblk))
        mpr_get_block_e(self.ctx, e)
        return e

    def block_energy(self, r: int) -> np.ndarray:
        E = np.zeros(self.nblk)
        mpr_block_energy(self.ctx, r, E)
        return E


class BatchFiller:
    """Many fields in one context (mpr_create_batch); numpy in, numpy out."""

    def __init__(self, values_list, mask_list, block: int, **options):
        self.values = [np.ascontiguousarray(v, dtype=np.float32) for v in values_list]
        self.masks = [np.ascontiguousarray(m, dtype=np.uint8) for m in mask_list]
        self.shapes = [m.shape for m in self.masks]
        self.opt = mpr_default_options(**options)
        self.ctx = mpr_create_batch([(h, w, block) for (h, w) in self.shapes], self.masks,
                                    self.values, self.opt)
        self.info = mpr_get_info(self.ctx)
        self.layout = mpr_get_slice_layout(self.ctx, len(self.shapes))

    def close(self):
        if getattr(self, "ctx", None):
            mpr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def calibrate(self) -> np.ndarray:
        T = np.zeros(self.info.nblk, np.float32)
        mpr_calibrate(self.ctx, T)
        return T

    def set_temperatures(self, T):
        mpr_set_temperatures(self.ctx, np.ascontiguousarray(T, dtype=np.float32))

    def energy_curve(self):
        return mpr_get_energy_curve(self.ctx)

    def sample_chains(self, n_chains: int, n_equil: int, n_samples: int):
        mpr_sample_chains(self.ctx, n_chains, n_equil, n_samples)

    def set_energy_curve(self, T, e):
        mpr_set_energy_curve(self.ctx, T, e)

    def simulate(self, n: int):
        mpr_simulate(self.ctx, n)

    def predict(self, truths=None):
        outs = [np.zeros(s, np.float32) for s in self.shapes]
        if truths is None:
            mpr_predict_batch(self.ctx, outs)
            return outs, None
        err = np.zeros(2 * len(outs), np.float64)
        mpr_predict_batch(self.ctx, outs,
                          [np.ascontiguousarray(t, dtype=np.float32) for t in truths], err)
        return outs, err.reshape(-1, 2)

    def block_slice(self, k: int, canvas_blocks: np.ndarray) -> np.ndarray:
        """The blocks of field k from a canvas-wide per-block array."""
        y0, x0, h, w = self.layout[k]
        lb = self.info.block
        grid = canvas_blocks.reshape(self.info.nby, self.info.nbx)
        return grid[y0 // lb:y0 // lb + (h + lb - 1) // lb,
                    x0 // lb:x0 // lb + (w + lb - 1) // lb].ravel()


def _check3(ctx, status: int):
    if status != MPR_OK:
        msg = load().mpr3_last_error(ctx).decode() if ctx else ""
        raise MprError(status, msg or load().mpr_status_string(status).decode())


class GapFiller3:
    """A D x H x W field (the 3-D extension); numpy in, numpy out."""

    def __init__(self, values, mask, block: int, **options):
        values = np.ascontiguousarray(values, dtype=np.float32)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.D, self.H, self.W = mask.shape
        self.opt = mpr_default_options(**options)
        out = C.c_void_p()
        g = mpr_grid3(self.D, self.H, self.W, block)
        st = load().mpr3_create(C.byref(g), _ptr(mask), _ptr(values), C.byref(self.opt),
                                C.byref(out))
        if st != MPR_OK:
            raise MprError(st, load().mpr_status_string(st).decode())
        self.ctx = out
        self.info = self.refresh()

    def profile(self) -> mpr_profile:
        p = mpr_profile()
        _check3(self.ctx, load().mpr3_get_profile(self.ctx, C.byref(p)))
        return p

    def refresh(self) -> mpr3_info:
        info = mpr3_info()
        _check3(self.ctx, load().mpr3_get_info(self.ctx, C.byref(info)))
        self.info = info
        return info

    @property
    def nblk(self) -> int:
        return self.info.nblk

    def close(self):
        if getattr(self, "ctx", None):
            load().mpr3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def block_stats(self):
        n = self.nblk
        Es, Nsp, Nb = np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32)
        ma, ng = np.zeros(n, np.float32), np.zeros(n, np.int32)
        _check3(self.ctx, load().mpr3_get_block_stats(self.ctx, _ptr(Es), _ptr(Nsp), _ptr(Nb),
                                                      _ptr(ma), _ptr(ng)))
        return Es, Nsp, Nb, ma, ng

    def calibrate(self) -> np.ndarray:
        T = np.zeros(self.nblk, np.float32)
        _check3(self.ctx, load().mpr3_calibrate(self.ctx, _ptr(T)))
        return T

    def set_temperatures(self, T):
        _check3(self.ctx, load().mpr3_set_temperatures(
            self.ctx, _ptr(np.ascontiguousarray(T, dtype=np.float32))))

    def simulate(self, n: int):
        _check3(self.ctx, load().mpr3_simulate(self.ctx, int(n)))

    def predict(self, truth=None):
        out = np.zeros((self.D, self.H, self.W), np.float32)
        err = np.zeros(2)
        tr = None if truth is None else np.ascontiguousarray(truth, dtype=np.float32)
        _check3(self.ctx, load().mpr3_predict(self.ctx, _ptr(out), _ptr(tr),
                                              None if tr is None else _ptr(err)))
        return out, (None if tr is None else (float(err[0]), float(err[1])))

    def sim_begin(self, n: int):
        _check3(self.ctx, load().mpr3_sim_begin(self.ctx, int(n)))

    def sim_end(self):
        _check3(self.ctx, load().mpr3_sim_end(self.ctx))

    def halfstep(self, colour: int, t: int, tag: int = 0):
        _check3(self.ctx, load().mpr3_halfstep(self.ctx, colour, t, tag))

    def get_state(self, r: int) -> np.ndarray:
        out = np.zeros((self.D, self.H, self.W), np.float32)
        _check3(self.ctx, load().mpr3_get_state(self.ctx, r, _ptr(out)))
        return out

    def set_state(self, r: int, angles):
        _check3(self.ctx, load().mpr3_set_state(
            self.ctx, r, _ptr(np.ascontiguousarray(angles, dtype=np.float32))))

