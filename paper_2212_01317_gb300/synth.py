"""Seeded synthetic inputs shaped like the remote-sensing grids of Lach & Zukovic
(arXiv 2212.01317, Sec. 3.1, Table 1): Gaussian random fields with exponential
covariance (stationary and with a correlation length that drifts across the
grid), optional nugget and lognormal marginal, thinned by uniformly random or
cloud-like (union of discs) gap masks (Sec. 3.2 thins the data at random).

This module produces values and masks only. It holds none of the method's
arithmetic (no transform, no energy, no sampling of the MPR chain), so both the
CUDA path and the CPU oracle can consume its output.

Recipe (each generator is a pure function of its arguments and seed):
  * GRF: spectral synthesis on a periodic torus of side max(L, 8*xi_max).
    C(r) = exp(-r/xi) with periodic distance, S = Re FFT(C) clipped at 0,
    field = Re IFFT(sqrt(S) * FFT(w)), w ~ N(0,1) white noise, cropped to HxW
    and standardised to zero mean / unit variance.
  * Non-stationary GRF: the same w filtered at 8 log-spaced xi_k; column x
    blends the two bracketing fields (linear weight in log xi) at
    xi(x) = xi_min + (xi_max - xi_min) * x / (W-1); re-standardised.
  * Random mask: exactly round(p*H*W) gap sites from a seeded permutation.
  * Disc mask: discs of uniform radius [r_min, r_max] and uniform centre are
    added one at a time until the gap fraction reaches the target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "grf", "grf_nonstationary", "mask_random", "mask_discs", "Workload",
    "workload", "WORKLOADS", "BatchWorkload", "batch_workload", "BATCH_WORKLOADS",
    "batch_sides", "batch_field", "batch_name",
]


def _torus_spectrum(n: int, xi: float) -> np.ndarray:
    d = np.arange(n, dtype=np.float64)
    d = np.minimum(d, n - d)
    r = np.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
    c = np.exp(-r / float(xi))
    s = np.fft.rfft2(c).real
    np.maximum(s, 0.0, out=s)
    return s


def _filtered(wf: np.ndarray, n: int, xi: float) -> np.ndarray:
    s = _torus_spectrum(n, xi)
    return np.fft.irfft2(np.sqrt(s) * wf, s=(n, n))


def _standardise(f: np.ndarray) -> np.ndarray:
    f = f - f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def grf(h: int, w: int, xi: float, seed: int) -> np.ndarray:
    """Stationary zero-mean unit-variance GRF with exponential covariance (float64)."""
    n = int(max(h, w, math.ceil(8 * xi)))
    rng = np.random.default_rng(seed)
    wn = rng.standard_normal((n, n))
    f = _filtered(np.fft.rfft2(wn), n, xi)[:h, :w]
    return _standardise(f)


def grf3(d: int, h: int, w: int, xi: float, seed: int) -> np.ndarray:
    """Stationary zero-mean unit-variance 3-D GRF with exponential covariance
    (spectral synthesis on a periodic cube of side max(d, h, w, 8 xi)), float64."""
    n = int(max(d, h, w, math.ceil(8 * xi)))
    ax = np.arange(n, dtype=np.float64)
    ax = np.minimum(ax, n - ax)
    r = np.sqrt(ax[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2)
    spec = np.fft.rfftn(np.exp(-r / float(xi))).real
    del r
    np.maximum(spec, 0.0, out=spec)
    rng = np.random.default_rng(seed)
    f = np.fft.irfftn(np.sqrt(spec) * np.fft.rfftn(rng.standard_normal((n, n, n))),
                      s=(n, n, n))[:d, :h, :w]
    return _standardise(f)


def grf_nonstationary(h: int, w: int, xi_min: float, xi_max: float, seed: int,
                      n_levels: int = 8) -> np.ndarray:
    """GRF whose correlation length grows linearly from xi_min (x=0) to xi_max (x=W-1)."""
    n = int(max(h, w, math.ceil(8 * xi_max)))
    rng = np.random.default_rng(seed)
    wn = rng.standard_normal((n, n))
    wf = np.fft.rfft2(wn)
    lx = np.linspace(math.log(xi_min), math.log(xi_max), n_levels)
    xis = np.exp(lx)
    x = np.arange(w, dtype=np.float64)
    xi_x = xi_min + (xi_max - xi_min) * x / max(w - 1, 1)
    lxi = np.log(xi_x)
    k = np.clip(np.searchsorted(lx, lxi, side="right") - 1, 0, n_levels - 2)
    a = np.clip((lxi - lx[k]) / (lx[k + 1] - lx[k]), 0.0, 1.0)
    out = np.zeros((h, w), dtype=np.float64)
    for lev in range(n_levels):
        wt = np.where(k == lev, 1.0 - a, 0.0) + np.where(k + 1 == lev, a, 0.0)
        if not np.any(wt):
            continue
        f = _standardise(_filtered(wf, n, xis[lev])[:h, :w])
        out += f * wt[None, :]
    return _standardise(out)


def mask_random(h: int, w: int, p: float, seed: int) -> np.ndarray:
    """uint8 mask (1 = gap) with exactly round(p*h*w) gaps."""
    n = h * w
    k = int(round(p * n))
    rng = np.random.default_rng(seed)
    m = np.zeros(n, dtype=np.uint8)
    m[rng.permutation(n)[:k]] = 1
    return m.reshape(h, w)


def mask_discs(h: int, w: int, frac: float, seed: int, r_min: float = 5.0,
               r_max: float = 60.0) -> np.ndarray:
    """uint8 mask (1 = gap): union of random discs until the gap fraction >= frac."""
    rng = np.random.default_rng(seed)
    m = np.zeros((h, w), dtype=np.uint8)
    target = frac * h * w
    covered = 0
    while covered < target:
        r = rng.uniform(r_min, r_max)
        cy = rng.uniform(0, h)
        cx = rng.uniform(0, w)
        y0, y1 = max(0, int(cy - r)), min(h, int(cy + r) + 1)
        x0, x1 = max(0, int(cx - r)), min(w, int(cx + r) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1)[:, None] + 0.5
        xx = np.arange(x0, x1)[None, :] + 0.5
        inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        sub = m[y0:y1, x0:x1]
        covered += int(np.count_nonzero(inside & (sub == 0)))
        sub[inside] = 1
    return m


@dataclass
class Workload:
    """One synthetic gap-filling problem: truth field, gap mask and run parameters."""
    name: str
    truth: np.ndarray          # float32 [H, W]
    mask: np.ndarray           # uint8 [H, W], 1 = gap
    block: int                 # l_b
    realizations: int
    storage: str = "f32"
    meta: dict = field(default_factory=dict)

    @property
    def values(self) -> np.ndarray:
        """Values handed to the library: truth at data sites, NaN at gaps."""
        v = self.truth.copy()
        v[self.mask != 0] = np.nan
        return v

    @property
    def shape(self):
        return self.truth.shape

    @property
    def n_gap(self) -> int:
        return int(np.count_nonzero(self.mask))


def _wl_field128(seed: int = 0) -> Workload:
    z = grf(128, 128, 8.0, seed).astype(np.float32)
    m = mask_random(128, 128, 0.33, seed + 1)
    return Workload("field128_xi8_p33_lb8_R10", z, m, 8, 10,
                    meta={"H": 128, "W": 128, "xi": 8, "p": 0.33})


def _wl_field1024(seed: int = 0) -> Workload:
    g = grf_nonstationary(1024, 1024, 4.0, 32.0, seed)
    rng = np.random.default_rng(seed + 7)
    z = (g + rng.normal(0.0, 0.1, g.shape)).astype(np.float32)
    m = mask_random(1024, 1024, 0.5, seed + 1)
    return Workload("field1024_xi4-32_nug0.1_p50_lb16_R100", z, m, 16, 100,
                    meta={"H": 1024, "W": 1024, "xi": [4, 32], "p": 0.5, "nugget": 0.1})


def _wl_field4096(seed: int = 0) -> Workload:
    g = grf_nonstationary(4096, 4096, 4.0, 64.0, seed)
    z = np.exp(0.5 * g).astype(np.float32)
    m = mask_discs(4096, 4096, 0.6, seed + 1)
    return Workload("field4096_xi4-64_lognormal_disc60_lb32", z, m, 32, 10, storage="bf16",
                    meta={"H": 4096, "W": 4096, "xi": [4, 64], "p": float(m.mean())})


def grf_nonstationary_gpu(h: int, w: int, xi_min: float, xi_max: float, seed: int,
                          n_levels: int = 8, device: str = "cuda") -> np.ndarray:
    """grf_nonstationary's recipe on the GPU (torch FFTs; white noise from a
    seeded torch generator, so the field differs from the numpy version's),
    for grids whose host FFTs would take minutes. float32 numpy [h, w]."""
    import torch
    n = int(max(h, w, math.ceil(8 * xi_max)))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    wf = torch.fft.rfft2(torch.randn((n, n), generator=gen, device=device))
    d = torch.arange(n, device=device, dtype=torch.float32)
    d = torch.minimum(d, n - d)
    lx = np.linspace(math.log(xi_min), math.log(xi_max), n_levels)
    x = np.arange(w, dtype=np.float64)
    lxi = np.log(xi_min + (xi_max - xi_min) * x / max(w - 1, 1))
    k = np.clip(np.searchsorted(lx, lxi, side="right") - 1, 0, n_levels - 2)
    a = np.clip((lxi - lx[k]) / (lx[k + 1] - lx[k]), 0.0, 1.0)
    out = torch.zeros((h, w), device=device, dtype=torch.float32)
    for lev in range(n_levels):
        wt = np.where(k == lev, 1.0 - a, 0.0) + np.where(k + 1 == lev, a, 0.0)
        if not np.any(wt):
            continue
        r = torch.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
        spec = torch.fft.rfft2(torch.exp(-r / float(np.exp(lx[lev])))).real.clamp_min_(0.0)
        del r
        f = torch.fft.irfft2(torch.sqrt(spec) * wf, s=(n, n))[:h, :w]
        del spec
        f = (f - f.mean()) / f.std()
        out += f * torch.as_tensor(wt, device=device, dtype=torch.float32)[None, :]
        del f
    out = (out - out.mean()) / out.std()
    return out.cpu().numpy()


def _wl_field16384(seed: int = 0) -> Workload:
    """16384^2 non-stationary GRF (xi 8 -> 128), 70 % disc gaps, l_b = 64, R = 20,
    BF16 state; generated on the GPU (needs CUDA)."""
    z = grf_nonstationary_gpu(16384, 16384, 8.0, 128.0, seed)
    m = mask_discs(16384, 16384, 0.7, seed + 1)
    return Workload("field16384_xi8-128_disc70_lb64_R20", z, m, 64, 20, storage="bf16",
                    meta={"H": 16384, "W": 16384, "xi": [8, 128], "p": float(m.mean())})


def _wl_cube256(seed: int = 0) -> Workload:
    """256^3 stationary 3-D GRF (xi = 8), 50 % random gaps, cubic blocks of side
    16, R = 20 (the 3-D extension)."""
    z = grf3(256, 256, 256, 8.0, seed).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    m = np.zeros(z.size, np.uint8)
    m[rng.permutation(z.size)[:z.size // 2]] = 1
    return Workload("cube256_xi8_p50_lb16_R20", z, m.reshape(z.shape), 16, 20,
                    meta={"D": 256, "H": 256, "W": 256, "xi": 8, "p": 0.5})


WORKLOADS = {
    "field128": _wl_field128,
    "cube256": _wl_cube256,
    "field1024": _wl_field1024,
    "field4096": _wl_field4096,
    "field16384": _wl_field16384,
}


def workload(name: str, seed: int = 0) -> Workload:
    return WORKLOADS[name](seed)


@dataclass
class BatchWorkload:
    """Many independent fields (time slices) filled together."""
    name: str
    truths: list               # float32 [H_k, W_k]
    masks: list                # uint8 [H_k, W_k], 1 = gap
    block: int
    realizations: int
    storage: str = "bf16"
    meta: dict = field(default_factory=dict)

    @property
    def n_gap(self) -> int:
        return int(sum(int(np.count_nonzero(m)) for m in self.masks))

    @property
    def n_sites(self) -> int:
        return int(sum(m.size for m in self.masks))


def _slice_params(n: int, seed: int) -> list:
    """Per-slice recipe of _slices: (side, xi, p, disc, field seed) for each of
    the n slices, drawn in order from one seeded generator (cheap: no field is
    generated)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(round(math.exp(rng.uniform(math.log(256), math.log(2048)))))
        xi = float(rng.uniform(4.0, 32.0))
        p = float(rng.uniform(0.1, 0.9))
        disc = bool(rng.uniform() < 0.5)
        out.append((L, xi, p, disc, seed * 1000003 + 17 * k))
    return out


def _slice_field(prm) -> tuple[np.ndarray, np.ndarray]:
    L, xi, p, disc, s = prm
    z = grf(L, L, xi, s).astype(np.float32)
    m = mask_discs(L, L, p, s + 1) if disc else mask_random(L, L, p, s + 1)
    return z, m


SLICES_BLOCK = 32        # temperature block side of the batch workloads
SLICES_R = 50            # realizations per field of the batch workloads


def _slices_name(n: int) -> str:
    return f"slices{n}_256-2048_xi4-32_p10-90_lb{SLICES_BLOCK}_R{SLICES_R}"


def _slices(n: int, seed: int) -> BatchWorkload:
    """n square slices, side round(exp(U(ln 256, ln 2048))), each its own seeded
    stationary GRF (xi ~ U(4, 32)), its own gap fraction p ~ U(0.1, 0.9), a
    uniformly random or disc mask with probability 1/2 each; l_b = 32, R = 50."""
    truths, masks, sides = [], [], []
    for prm in _slice_params(n, seed):
        z, m = _slice_field(prm)
        truths.append(z)
        masks.append(m)
        sides.append(prm[0])
    return BatchWorkload(_slices_name(n), truths, masks, SLICES_BLOCK, SLICES_R,
                         meta={"slices": n, "sides": [min(sides), max(sides)],
                               "sites": int(sum(x * x for x in sides))})


def batch_sides(name: str, seed: int = 0) -> list:
    """Field sides of a batch workload, without generating its fields."""
    n = _BATCH_SIZES[name]
    return [prm[0] for prm in _slice_params(n, seed)]


def batch_field(name: str, k: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(truth, mask) of field k of a batch workload, generated alone (the same
    arrays batch_workload(name, seed) holds at position k)."""
    n = _BATCH_SIZES[name]
    return _slice_field(_slice_params(n, seed)[k])


def batch_name(name: str) -> str:
    return _slices_name(_BATCH_SIZES[name])


_BATCH_SIZES = {"slices256": 256, "slices32": 32}

BATCH_WORKLOADS = {
    "slices256": lambda seed=0: _slices(256, seed),
    "slices32": lambda seed=0: _slices(32, seed),
}


def batch_workload(name: str, seed: int = 0) -> BatchWorkload:
    return BATCH_WORKLOADS[name](seed)


def small_problem(h: int, w: int, p: float, seed: int, xi: float = 6.0,
                  kind: str = "random") -> tuple[np.ndarray, np.ndarray]:
    """(truth float32 [h,w], mask uint8 [h,w]) for tests at arbitrary small sizes."""
    z = grf(h, w, xi, seed).astype(np.float32)
    if kind == "random":
        m = mask_random(h, w, p, seed + 1)
    else:
        m = mask_discs(h, w, p, seed + 1, r_min=1.5, r_max=max(2.0, min(h, w) / 6))
    return z, m
