"""CPU oracle for SV-MPR gap filling (Lach & Zukovic, arXiv 2212.01317).

TEST INFRASTRUCTURE ONLY. A plain FP64 C restatement of the method
(``mpr_oracle.c``) plus this ctypes wrapper. Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the library under
``paper_2212_01317_gb300`` never does and shares no code with it.

Every function here is argument marshalling around the C code, except
``gapfill`` which strings the C steps together in the paper's order
(transform, block statistics, calibration, realizations, mean,
back-transform).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TWO_PI = 2.0 * np.pi


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, no FP contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "mpr_oracle.h")))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Model(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("lb", C.c_int32),
                ("nbx", C.c_int32), ("nby", C.c_int32), ("nblk", C.c_int32),
                ("q", C.c_double), ("J", C.c_double),
                ("key0", C.c_uint32), ("key1", C.c_uint32),
                ("overrelax", C.c_int32), ("K", C.c_int32), ("threads", C.c_int32),
                ("T_site", C.c_void_p), ("D", C.c_int32), ("nbz", C.c_int32),
                ("storage", C.c_int32), ("stop_rule", C.c_int32), ("n_fit", C.c_int32),
                ("n_f", C.c_int32)]


class Diag(C.Structure):
    _fields_ = [("dE", C.c_double), ("theta", C.c_double), ("phi_or", C.c_double),
                ("R", C.c_double), ("phi_old", C.c_double), ("phi_prop", C.c_double),
                ("accepted", C.c_int32), ("or_applied", C.c_int32)]


DIAG_DTYPE = np.dtype([("dE", "f8"), ("theta", "f8"), ("phi_or", "f8"), ("R", "f8"),
                       ("phi_old", "f8"), ("phi_prop", "f8"), ("accepted", "i4"),
                       ("or_applied", "i4")])
assert DIAG_DTYPE.itemsize == C.sizeof(Diag)

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        MP = C.POINTER(Model)
        sig = {
            "orc_model_init": (None, [MP, i32, i32, i32, f64, f64, u64, u32]),
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_u01": (f64, [u32]),
            "orc_round_store": (f64, [f64, i32]),
            "orc_site_uniforms": (None, [MP, i64, u32, u32, u32, P, P]),
            "orc_transform": (C.c_int, [i64, P, P, P, P, P]),
            "orc_backtransform": (None, [i64, P, P, P, f64, f64, P]),
            "orc_block_stats": (None, [MP, P, P, P, P, P, P, P, P, P]),
            "orc_block_energy": (None, [MP, P, P]),
            "orc_total_energy": (f64, [MP, P]),
            "orc_update_site": (None, [MP, P, P, i64, f64, u32, u32, u32, P]),
            "orc_halfstep": (None, [MP, P, P, C.c_int, P, P, u32, u32, u32, P]),
            "orc_init_block_mean": (None, [MP, P, P, P, P, f64]),
            "orc_init_random": (None, [MP, P, P, u32]),
            "orc_simulate_one": (C.c_int, [MP, P, P, P, P, P, P, P, i32, u32, P, P]),
            "orc_stop_init": (None, [MP, P, P, P, P, P, P, P, P]),
            "orc_stop_update": (C.c_int, [MP, i32, i32, P, P, P, P, P, P, P]),
            "orc_stop_update_window": (C.c_int, [MP, i32, i32, P, P, P, P, P, P]),
            "orc_window_slope": (f64, [MP, i32, P, C.c_int]),
            "orc_calibrate": (None, [MP, P, P, P, P, P, i32, i32, i32, i32, f64, f64, P, P]),
            "orc_median_targeted": (f64, [i32, P, P]),
            "orc_scores": (None, [i64, P, P, P, P, P]),
            "orc_sst_temperatures": (None, [MP, P, i32, i32, P]),
            "orc_calibrate_points": (None, [MP, P, P, P, P, P, i32, i32, i32, i32, i32, f64, f64,
                                            P, f64, i32, P, P, P]),
            "orc_sample_chain": (None, [MP, P, P, P, i32, i32, u32, P]),
            "orc_energy_curve": (None, [f64, f64, u64, i32, i32, i32, P, i32, i32, P]),
            "orc_curve_T0": (f64, [i32, P, P, f64]),
            "orc3_model_init": (None, [MP, i32, i32, i32, i32, f64, f64, u64, u32]),
            "orc3_block_stats": (None, [MP, P, P, P, P, P, P, P, P, P]),
            "orc3_block_energy": (None, [MP, P, P]),
            "orc3_update_site": (None, [MP, P, P, i64, f64, u32, u32, u32, P]),
            "orc3_halfstep": (None, [MP, P, P, C.c_int, P, P, u32, u32, u32, P]),
            "orc3_init_block_mean": (None, [MP, P, P, P, P, f64]),
            "orc3_simulate_one": (C.c_int, [MP, P, P, P, P, P, P, P, i32, u32, P, P]),
            "orc3_calibrate": (None, [MP, P, P, P, P, P, i32, i32, i32, i32, f64, f64, P]),
            "orc_energy_moments": (None, [MP, P, P, P, i32, i32, i32, u32, P, P, P, P, P]),
            "orc_calibrate_newton": (None, [MP, P, P, P, P, P, i32, i32, i32, i32, f64, f64, f64,
                                            P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def round_store(v: float, storage: int) -> float:
    """v rounded to the stored angle type (0 exact, 1 BF16, 2 FP16) via FP32."""
    return lib().orc_round_store(float(v), int(storage))


@dataclass
class BlockStats:
    Es: np.ndarray
    Nsp: np.ndarray
    Nb: np.ndarray
    mean_angle: np.ndarray
    n_gap: np.ndarray
    n_sample: np.ndarray
    global_mean: float

    @property
    def es(self) -> np.ndarray:
        out = np.zeros_like(self.Es)
        t = self.Nsp > 0
        out[t] = self.Es[t] / self.Nsp[t]
        return out


class Oracle:
    """One grid geometry + model parameters; methods mirror the C functions."""

    def __init__(self, H: int, W: int, lb: int, q: float = 0.5, J: float = 1.0,
                 seed: int = 0, slice_id: int = 0, overrelax: bool = True, K: int = 0,
                 threads: int = 0, storage: int = 0, stop_rule: int = 0, n_fit: int = 20,
                 n_f: int = 5):
        self.m = Model()
        lib().orc_model_init(C.byref(self.m), H, W, lb, q, J, seed & (2**64 - 1), slice_id)
        self.m.overrelax = 1 if overrelax else 0
        self.m.K = int(K)
        self.m.threads = int(threads)
        self.m.storage = int(storage)     # 0 exact, 1 BF16, 2 FP16 stored gap angles
        self.m.stop_rule = int(stop_rule)  # 0 CROSS, 1 WINDOW (Sec. 3.4 n_fit, n_f)
        self.m.n_fit = int(n_fit)
        self.m.n_f = int(n_f)
        self.H, self.W, self.lb = H, W, lb

    @property
    def nblk(self) -> int:
        return self.m.nblk

    @property
    def nbx(self) -> int:
        return self.m.nbx

    def block_index(self) -> np.ndarray:
        y, x = np.mgrid[0:self.H, 0:self.W]
        return (y // self.lb) * self.m.nbx + x // self.lb

    def site_uniforms(self, i: int, t: int, tag: int, r: int):
        u0, u1 = C.c_double(), C.c_double()
        lib().orc_site_uniforms(C.byref(self.m), i, t, tag, r, C.byref(u0), C.byref(u1))
        return u0.value, u1.value

    @staticmethod
    def transform(values: np.ndarray, mask: np.ndarray):
        v = np.ascontiguousarray(values, dtype=np.float32).ravel()
        mk = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
        phi = np.zeros(v.size, dtype=np.float64)
        zmin, zmax = C.c_double(), C.c_double()
        deg = lib().orc_transform(v.size, _p(v), _p(mk), C.byref(zmin), C.byref(zmax), _p(phi))
        return phi.reshape(np.shape(values)), zmin.value, zmax.value, bool(deg)

    @staticmethod
    def backtransform(mean_phi, mask, values, zmin, zmax) -> np.ndarray:
        mp = np.ascontiguousarray(mean_phi, dtype=np.float64).ravel()
        mk = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
        v = np.ascontiguousarray(values, dtype=np.float32).ravel()
        out = np.zeros(mp.size, dtype=np.float32)
        lib().orc_backtransform(mp.size, _p(mp), _p(mk), _p(v), zmin, zmax, _p(out))
        return out.reshape(np.shape(mean_phi))

    def block_stats(self, phi, mask) -> BlockStats:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        n = self.nblk
        Es = np.zeros(n); Nsp = np.zeros(n, np.int64); Nb = np.zeros(n, np.int64)
        ma = np.zeros(n); ng = np.zeros(n, np.int64); ns = np.zeros(n, np.int64)
        gm = C.c_double()
        lib().orc_block_stats(C.byref(self.m), _p(ph), _p(mk), _p(Es), _p(Nsp), _p(Nb), _p(ma),
                              _p(ng), _p(ns), C.byref(gm))
        return BlockStats(Es, Nsp, Nb, ma, ng, ns, gm.value)

    def block_energy(self, phi) -> np.ndarray:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        E = np.zeros(self.nblk)
        lib().orc_block_energy(C.byref(self.m), _p(ph), _p(E))
        return E

    def total_energy(self, phi) -> float:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        return lib().orc_total_energy(C.byref(self.m), _p(ph))

    def sst_temperatures(self, T_blk, r_s: int, n_s: int) -> np.ndarray:
        """Sec. 2.2.3 site temperatures from the block temperatures."""
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        out = np.zeros((self.H, self.W))
        lib().orc_sst_temperatures(C.byref(self.m), _p(T), int(r_s), int(n_s), _p(out))
        return out

    def use_site_temperatures(self, T_site):
        """Updates take T from T_site[H, W] (SST) instead of the block's T; None
        restores the block temperatures (BST). The array is kept alive here."""
        if T_site is None:
            self._T_site = None
            self.m.T_site = None
            return
        self._T_site = np.ascontiguousarray(T_site, dtype=np.float64).reshape(self.H, self.W)
        self.m.T_site = self._T_site.ctypes.data

    def update_site(self, phi: np.ndarray, mask, i: int, T: float, t: int, tag: int, r: int):
        """Update site i of phi (float64, modified in place); returns the diagnostics."""
        assert phi.dtype == np.float64 and phi.flags.c_contiguous
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        d = Diag()
        lib().orc_update_site(C.byref(self.m), _p(phi), _p(mk), i, T, t, tag, r, C.byref(d))
        return d

    def halfstep(self, phi: np.ndarray, mask, colour: int, T_blk, active=None, t: int = 1,
                 tag: int = 0, r: int = 0, diag: bool = False):
        """In-place half-step on phi (float64 C-contiguous). Returns diag array or None."""
        assert phi.dtype == np.float64 and phi.flags.c_contiguous
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        dg = np.zeros(phi.size, dtype=DIAG_DTYPE) if diag else None
        if dg is not None:
            dg["phi_or"] = np.nan
        lib().orc_halfstep(C.byref(self.m), _p(phi), _p(mk), colour, _p(T),
                           None if act is None else _p(act), t, tag, r,
                           None if dg is None else _p(dg))
        return dg

    def init_block_mean(self, phi, mask, st: BlockStats) -> np.ndarray:
        out = np.ascontiguousarray(phi, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        lib().orc_init_block_mean(C.byref(self.m), _p(out), _p(mk), _p(st.mean_angle),
                                  _p(st.n_sample), st.global_mean)
        return out

    def init_random(self, phi, mask, r: int) -> np.ndarray:
        out = np.ascontiguousarray(phi, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        lib().orc_init_random(C.byref(self.m), _p(out), _p(mk), r)
        return out

    def stop_init(self, E0, st: BlockStats):
        n = self.nblk
        sigma = np.zeros(n, np.int8); active = np.zeros(n, np.uint8); stop = np.zeros(n, np.int32)
        E0 = np.ascontiguousarray(E0, dtype=np.float64)
        lib().orc_stop_init(C.byref(self.m), _p(E0), _p(st.Es), _p(st.Nsp), _p(st.Nb),
                            _p(st.n_gap), _p(sigma), _p(active), _p(stop))
        return sigma, active, stop

    def stop_update(self, t, n_max, E, st: BlockStats, sigma, active, stop) -> int:
        E = np.ascontiguousarray(E, dtype=np.float64)
        return lib().orc_stop_update(C.byref(self.m), t, n_max, _p(E), _p(st.Es), _p(st.Nsp),
                                     _p(st.Nb), _p(sigma), _p(active), _p(stop))

    def stop_update_window(self, t, n_max, st: BlockStats, sigma, hist, active, stop) -> int:
        """hist: [n_fit, nblk] ring of e_b by sweep mod n_fit (e_b(t) written)."""
        hist = np.ascontiguousarray(hist, dtype=np.float64)
        return lib().orc_stop_update_window(C.byref(self.m), t, n_max, _p(st.Es), _p(st.Nsp),
                                            _p(sigma), _p(hist), _p(active), _p(stop))

    def window_slope(self, t, hist, b) -> float:
        hist = np.ascontiguousarray(hist, dtype=np.float64)
        return lib().orc_window_slope(C.byref(self.m), t, _p(hist), int(b))

    def simulate_one(self, phi0, mask, T_blk, st: BlockStats, n_max: int, r: int,
                     trace: bool = False):
        phi = np.ascontiguousarray(phi0, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        stop = np.zeros(self.nblk, np.int32)
        tr = np.full((n_max + 1, self.nblk), np.nan) if trace else None
        n = lib().orc_simulate_one(C.byref(self.m), _p(phi), _p(mk), _p(T), _p(st.Es),
                                   _p(st.Nsp), _p(st.Nb), _p(st.n_gap), n_max, r, _p(stop),
                                   None if tr is None else _p(tr))
        return phi, stop, n, tr

    def sample_chain(self, phi0, mask, T_blk, n_equil: int, n_samples: int, r: int,
                     sum_out=None) -> np.ndarray:
        """Sampling variant: the chain's states after sweeps n_equil + 1 ..
        n_equil + n_samples summed at the gap sites (added to sum_out)."""
        ph = np.ascontiguousarray(phi0, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        out = np.zeros(self.H * self.W) if sum_out is None else sum_out
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.H * self.W
        lib().orc_sample_chain(C.byref(self.m), _p(ph), _p(mk), _p(T), int(n_equil),
                               int(n_samples), int(r), _p(out))
        return out

    def calibrate(self, phi_init, mask, st: BlockStats, n_eq=25, n_meas=20, n_bisect=24,
                  chains=1, T_lo=1e-4, T_hi=2.0, trace=False):
        ph = np.ascontiguousarray(phi_init, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.zeros(self.nblk)
        tr = np.zeros((n_bisect, self.nblk)) if trace else None
        lib().orc_calibrate(C.byref(self.m), _p(ph), _p(mk), _p(st.Es), _p(st.Nsp), _p(st.Nb),
                            n_eq, n_meas, n_bisect, chains, T_lo, T_hi, _p(T),
                            None if tr is None else _p(tr))
        return (T, tr) if trace else T

    def energy_moments(self, phi_chains, mask, T_blk, n_eq: int, n_meas: int, tag: int,
                       st: BlockStats):
        """Moments of the block energies over the chains' measured sweeps; the
        chains' states phi_chains[chains, H, W] advance in place. Returns
        (mean_e, var_E, cov_right, cov_down), each nblk long."""
        assert phi_chains.dtype == np.float64 and phi_chains.flags.c_contiguous
        chains = phi_chains.shape[0]
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        out = [np.zeros(self.nblk) for _ in range(4)]
        lib().orc_energy_moments(C.byref(self.m), _p(phi_chains), _p(mk), _p(T), n_eq, n_meas,
                                 chains, tag, _p(st.Nb), *[_p(a) for a in out])
        return tuple(out)

    def calibrate_newton(self, phi_init, mask, st: BlockStats, n_eq=25, n_meas=20, n_newton=6,
                         chains=1, T_lo=1e-4, T_hi=2.0, T0=0.1, trace=False):
        ph = np.ascontiguousarray(phi_init, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.zeros(self.nblk)
        tr = np.zeros((n_newton, self.nblk)) if trace else None
        lib().orc_calibrate_newton(C.byref(self.m), _p(ph), _p(mk), _p(st.Es), _p(st.Nsp),
                                   _p(st.Nb), n_eq, n_meas, n_newton, chains, T_lo, T_hi, T0,
                                   _p(T), None if tr is None else _p(tr))
        return (T, tr) if trace else T

    def calibrate_points(self, phi_init, mask, st: BlockStats, n_eq=25, n_meas=20, n_iter=16,
                         chains=1, points=2, T_lo=1e-4, T_hi=2.0, T0_warm=None, warm=1.5,
                         trace=False, n_eq_next=-1):
        """k-point calibration; T0_warm (per block, from curve_T0) starts the
        first iteration's points on [T0 / warm, T0 * warm]. n_eq_next >= 0
        keeps every chain's state across iterations (n_eq_next equilibration
        sweeps after the first iteration). trace=True also
        returns the per-iteration mean e_b and temperatures of every point,
        each [n_iter, points, nblk]."""
        ph = np.ascontiguousarray(phi_init, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.zeros(self.nblk)
        t0 = None if T0_warm is None else np.ascontiguousarray(T0_warm, dtype=np.float64)
        et = np.zeros((n_iter, points, self.nblk)) if trace else None
        pt = np.zeros((n_iter, points, self.nblk)) if trace else None
        lib().orc_calibrate_points(C.byref(self.m), _p(ph), _p(mk), _p(st.Es), _p(st.Nsp),
                                   _p(st.Nb), n_eq, n_meas, n_iter, chains, points, T_lo, T_hi,
                                   None if t0 is None else _p(t0), float(warm),
                                   int(n_eq_next), _p(T),
                                   None if et is None else _p(et), None if pt is None else _p(pt))
        return (T, et, pt) if trace else T

    def warm_T0(self, st: BlockStats, T_curve, e_curve) -> np.ndarray:
        """Per-block T0 = curve_T0(e_s,b) (0 for blocks without sample bonds)."""
        es = st.es
        return np.array([curve_T0(T_curve, e_curve, es[b]) if st.Nsp[b] > 0 else 0.0
                         for b in range(self.nblk)])

    @staticmethod
    def median_targeted(T, Nsp) -> float:
        T = np.ascontiguousarray(T, dtype=np.float64)
        Nsp = np.ascontiguousarray(Nsp, dtype=np.int64)
        return lib().orc_median_targeted(T.size, _p(T), _p(Nsp))

    @staticmethod
    def scores(pred, truth, mask):
        p = np.ascontiguousarray(pred, dtype=np.float32).ravel()
        t = np.ascontiguousarray(truth, dtype=np.float32).ravel()
        mk = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
        a, r = C.c_double(), C.c_double()
        lib().orc_scores(p.size, _p(p), _p(t), _p(mk), C.byref(a), C.byref(r))
        return a.value, r.value


def energy_curve(T, L: int = 64, n_eq: int = 25, n_meas: int = 20, seed: int = 0,
                 q: float = 0.5, J: float = 1.0, overrelax: bool = True) -> np.ndarray:
    """Unconditional e(T) of a data-free L x L lattice (orc_energy_curve)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    e = np.zeros(T.size)
    lib().orc_energy_curve(q, J, seed & (2**64 - 1), 1 if overrelax else 0, L, T.size, _p(T),
                           n_eq, n_meas, _p(e))
    return e


def curve_T0(T, e, e_s: float) -> float:
    """T where the non-decreasing envelope of the curve reaches e_s."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    return lib().orc_curve_T0(T.size, _p(T), _p(e), float(e_s))


class Oracle3:
    """A D x H x W grid (6-neighbour bonds, cubic blocks); arrays are [D, H, W]."""

    def __init__(self, D: int, H: int, W: int, lb: int, q: float = 0.5, J: float = 1.0,
                 seed: int = 0, slice_id: int = 0, overrelax: bool = True):
        self.m = Model()
        lib().orc3_model_init(C.byref(self.m), D, H, W, lb, q, J, seed & (2**64 - 1), slice_id)
        self.m.overrelax = 1 if overrelax else 0
        self.D, self.H, self.W, self.lb = D, H, W, lb

    @property
    def nblk(self) -> int:
        return self.m.nblk

    def block_index(self) -> np.ndarray:
        z, y, x = np.mgrid[0:self.D, 0:self.H, 0:self.W]
        lb = self.lb
        return ((z // lb) * self.m.nby + y // lb) * self.m.nbx + x // lb

    def block_stats(self, phi, mask) -> BlockStats:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        n = self.nblk
        Es = np.zeros(n); Nsp = np.zeros(n, np.int64); Nb = np.zeros(n, np.int64)
        ma = np.zeros(n); ng = np.zeros(n, np.int64); ns = np.zeros(n, np.int64)
        gm = C.c_double()
        lib().orc3_block_stats(C.byref(self.m), _p(ph), _p(mk), _p(Es), _p(Nsp), _p(Nb), _p(ma),
                               _p(ng), _p(ns), C.byref(gm))
        return BlockStats(Es, Nsp, Nb, ma, ng, ns, gm.value)

    def block_energy(self, phi) -> np.ndarray:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        E = np.zeros(self.nblk)
        lib().orc3_block_energy(C.byref(self.m), _p(ph), _p(E))
        return E

    def update_site(self, phi: np.ndarray, mask, i: int, T: float, t: int, tag: int, r: int):
        assert phi.dtype == np.float64 and phi.flags.c_contiguous
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        d = Diag()
        lib().orc3_update_site(C.byref(self.m), _p(phi), _p(mk), i, T, t, tag, r, C.byref(d))
        return d

    def halfstep(self, phi: np.ndarray, mask, colour: int, T_blk, active=None, t: int = 1,
                 tag: int = 0, r: int = 0, diag: bool = False):
        assert phi.dtype == np.float64 and phi.flags.c_contiguous
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        dg = np.zeros(phi.size, dtype=DIAG_DTYPE) if diag else None
        if dg is not None:
            dg["phi_or"] = np.nan
        lib().orc3_halfstep(C.byref(self.m), _p(phi), _p(mk), colour, _p(T),
                            None if act is None else _p(act), t, tag, r,
                            None if dg is None else _p(dg))
        return dg

    def init_block_mean(self, phi, mask, st: BlockStats) -> np.ndarray:
        ph = np.ascontiguousarray(phi, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        lib().orc3_init_block_mean(C.byref(self.m), _p(ph), _p(mk), _p(st.mean_angle),
                                   _p(st.n_sample), st.global_mean)
        return ph

    def simulate_one(self, phi0, mask, T_blk, st: BlockStats, n_max: int, r: int):
        phi = np.ascontiguousarray(phi0, dtype=np.float64).copy()
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.ascontiguousarray(T_blk, dtype=np.float64)
        stop = np.zeros(self.nblk, np.int32)
        n = lib().orc3_simulate_one(C.byref(self.m), _p(phi), _p(mk), _p(T), _p(st.Es),
                                    _p(st.Nsp), _p(st.Nb), _p(st.n_gap), n_max, r, _p(stop), None)
        return phi, stop, n

    def calibrate(self, phi_init, mask, st: BlockStats, n_eq=25, n_meas=20, n_bisect=24,
                  chains=1, T_lo=1e-4, T_hi=2.0):
        ph = np.ascontiguousarray(phi_init, dtype=np.float64)
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        T = np.zeros(self.nblk)
        lib().orc3_calibrate(C.byref(self.m), _p(ph), _p(mk), _p(st.Es), _p(st.Nsp), _p(st.Nb),
                             n_eq, n_meas, n_bisect, chains, T_lo, T_hi, _p(T))
        return T


def gapfill3(values, mask, lb: int, R: int, seed: int = 0, slice_id: int = 0, n_max: int = 200,
             n_eq: int = 25, n_meas: int = 20, n_bisect: int = 24, chains: int = 1, T_blk=None):
    """The method on a D x H x W grid (Sec. 2.1 transform, Eq. 2 per cubic block,
    calibration, R local-equilibrium realizations, mean, back-transform)."""
    values = np.asarray(values, dtype=np.float32)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    D, H, W = mask.shape
    o = Oracle3(D, H, W, lb, seed=seed, slice_id=slice_id)
    phi, zmin, zmax, _ = Oracle.transform(values.reshape(D * H, W), mask.reshape(D * H, W))
    phi = phi.reshape(D, H, W)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    T = o.calibrate(phi0, mask, st, n_eq, n_meas, n_bisect, chains) if T_blk is None else \
        np.asarray(T_blk, dtype=np.float64)
    acc = np.zeros((D, H, W))
    updates = 0
    for k in range(R):
        ph, stop, _ = o.simulate_one(phi0, mask, T, st, n_max, k)
        acc += ph
        updates += int(np.sum(stop.astype(np.int64) * st.n_gap))
    mean_phi = acc / R if R > 0 else phi0
    pred = Oracle.backtransform(mean_phi.reshape(D * H, W), mask.reshape(D * H, W),
                                values.reshape(D * H, W), zmin, zmax).reshape(D, H, W)
    return GapfillResult(pred, T, None, None, mean_phi, zmin, zmax, st, updates)


@dataclass
class GapfillResult:
    pred: np.ndarray
    T: np.ndarray
    stop_sweeps: np.ndarray      # [R, nblk]
    sweeps: np.ndarray           # [R]
    mean_phi: np.ndarray
    zmin: float
    zmax: float
    stats: BlockStats
    gap_updates: int


def gapfill(values, mask, lb: int, R: int, seed: int = 0, slice_id: int = 0, q: float = 0.5,
            J: float = 1.0, n_max: int = 200, n_eq: int = 25, n_meas: int = 20,
            n_bisect: int = 24, chains: int = 1, T_lo: float = 1e-4, T_hi: float = 2.0,
            T_blk=None, overrelax: bool = True, threads: int = 0,
            r0: int = 0, sst=None, stop_rule: int = 0, n_fit: int = 20,
            n_f: int = 5) -> GapfillResult:
    """The whole method on the CPU: Sec. 2.1 transform, Eq. 2 per block,
    per-block T by energy matching (Sec. 2.2.2; skipped when T_blk is given),
    R local-equilibrium realizations from the block-mean start (Sec. 3.3.3,
    Sec. 3.4), their mean and the back-transform (Sec. 2.1, Sec. 3.2).
    sst = (r_s, n_s): the realizations run at the smoothed site temperatures
    of Sec. 2.2.3 instead of the block temperatures."""
    values = np.asarray(values, dtype=np.float32)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = mask.shape
    o = Oracle(H, W, lb, q=q, J=J, seed=seed, slice_id=slice_id, overrelax=overrelax,
               threads=threads, stop_rule=stop_rule, n_fit=n_fit, n_f=n_f)
    phi, zmin, zmax, deg = o.transform(values, mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    if T_blk is None:
        T = o.calibrate(phi0, mask, st, n_eq, n_meas, n_bisect, chains, T_lo, T_hi)
    else:
        T = np.asarray(T_blk, dtype=np.float64)
    if sst is not None:
        o.use_site_temperatures(o.sst_temperatures(T, sst[0], sst[1]))
    acc = np.zeros((H, W))
    stops = np.zeros((R, o.nblk), np.int32)
    sweeps = np.zeros(R, np.int32)
    updates = 0
    for k in range(R):
        ph, stop, n, _ = o.simulate_one(phi0, mask, T, st, n_max, r0 + k)
        acc += ph
        stops[k] = stop
        sweeps[k] = n
        updates += int(np.sum(stop.astype(np.int64) * st.n_gap))
    mean_phi = acc / R if R > 0 else phi0
    pred = o.backtransform(mean_phi, mask, values, zmin, zmax)
    return GapfillResult(pred, T, stops, sweeps, mean_phi, zmin, zmax, st, updates)
