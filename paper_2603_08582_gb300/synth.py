"""Seeded synthetic inputs for the online sparse-SAR workloads.

This module only draws random numbers and lays out the experiment geometry
(platform track, scene coefficients, noise draws, Gaussian dictionary).  It
holds none of the reconstruction arithmetic: no phase synthesis, no Gram or
data-vector update, no FISTA step.  Both the CUDA library (through its Python
binding) and the FP64 oracle consume what it produces.

The Gaussian dictionary is defined by a counter-based generator,
Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011), followed by a Box-Muller transform and unit-norm
column scaling.  The CUDA library implements the same published definition on
the device so that a 16384 x 32768 dictionary never has to cross PCIe/C2C;
this module implements it on the host so that the oracle sees identical atoms.

Workload recipes (the paper's own scenes exist only as missing figures, so
these stand in for them):

* track: circular aperture centred on the scene centre, horizontal radius r,
  altitude h, P pulses evenly spaced (both ends inclusive) over `span_deg`
  starting at azimuth 0 (§II, Eq. 3 uses gamma(s_n) only through ranges).
* pixel grid: nx x ny pixels of `pixel_m` metres, centred at the origin, on
  flat ground (Psi = 0, §II).
* scene: k = round(frac * M) nonzero coefficients at distinct uniformly drawn
  positions, |a| ~ U(0.5, 1), arg a ~ U[0, 2 pi).  The clustered variant puts
  3 x 3 pixel blocks around round(frac * N) uniformly drawn centres.
* noise: unit complex Gaussian draws w_s in C^K; the per-pulse scale that
  sets the SNR is applied by `scale_noise`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np

SPEED_OF_LIGHT = 299_792_458.0

# --------------------------------------------------------------------------
# Workload definitions
# --------------------------------------------------------------------------


@dataclass
class Workload:
    """One online SAR workload: grid, band, track, scene and solver knobs."""

    name: str
    nx: int
    ny: int
    n_freq: int
    f_lo_hz: float
    f_hi_hz: float
    n_pulses: int
    span_deg: float
    radius_m: float = 1000.0
    height_m: float = 500.0
    pixel_m: float = 1.0
    theta0_deg: float = 0.0
    dictionary: str = "identity"     # "identity" | "gaussian" | "edgelet"
    n_atoms: Optional[int] = None    # None => M = N
    edgelet_lengths: tuple = ()      # edgelet atoms: lengths x angles x pixels
    edgelet_angles: tuple = ()       # degrees, multiples of 45
    dict_seed: int = 0
    sparsity: float = 0.05
    clustered: bool = False
    snr_db: float = 20.0
    inner_steps: int = 20            # m of Algorithm 1
    lambda_rel: float = 0.05         # lambda_n = lambda_rel * ||b_n||_inf
    tol: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny

    @property
    def m_atoms(self) -> int:
        if self.dictionary == "edgelet":
            return len(self.edgelet_lengths) * len(self.edgelet_angles) * self.n_pixels
        return self.n_atoms if self.n_atoms is not None else self.n_pixels

    def as_dict(self) -> dict:
        return asdict(self)


def workloads() -> dict:
    """The five configurations of the online SAR hot path, by name."""
    return {
        # plain FP64 method, pixel basis
        "c1_32x32_fp64": Workload(
            name="c1_32x32_fp64", nx=32, ny=32, n_freq=128,
            f_lo_hz=9.9e9, f_hi_hz=10.1e9, n_pulses=64, span_deg=30.0,
            sparsity=0.05, snr_db=20.0, inner_steps=20, seed=1),
        # precision form, overcomplete Gaussian dictionary (M = 2N)
        "c2_128x128_split_bf16": Workload(
            name="c2_128x128_split_bf16", nx=128, ny=128, n_freq=512,
            f_lo_hz=9.75e9, f_hi_hz=10.25e9, n_pulses=256, span_deg=45.0,
            dictionary="gaussian", n_atoms=2 * 128 * 128, dict_seed=2,
            sparsity=0.03, snr_db=25.0, inner_steps=20, tol=1e-4, seed=2),
        # differentiation form
        "c3_64x64_adjoint": Workload(
            name="c3_64x64_adjoint", nx=64, ny=64, n_freq=256,
            f_lo_hz=9.75e9, f_hi_hz=10.25e9, n_pulses=128, span_deg=30.0,
            sparsity=0.04, snr_db=20.0, inner_steps=64, seed=3,
            extra={"unroll_T": 64, "checkpoint_every": 8}),
        # large online form
        "c5_256x256_split_bf16": Workload(
            name="c5_256x256_split_bf16", nx=256, ny=256, n_freq=1024,
            f_lo_hz=9.5e9, f_hi_hz=10.5e9, n_pulses=1024, span_deg=60.0,
            sparsity=0.01, clustered=True, snr_db=15.0, inner_steps=10,
            seed=5),
    }


def batch_workloads(n_scenes: int = 96, seed: int = 4) -> list:
    """Batching form: uneven scenes, each with its own random track."""
    rng = np.random.default_rng(seed)
    sides = [32, 48, 64, 80, 96]
    out = []
    for i in range(n_scenes):
        side = int(rng.choice(sides))
        out.append(Workload(
            name=f"c4_scene{i:03d}_{side}x{side}", nx=side, ny=side,
            n_freq=256, f_lo_hz=9.9e9, f_hi_hz=10.1e9,
            n_pulses=int(rng.integers(64, 193)),
            span_deg=float(rng.uniform(20.0, 40.0)),
            radius_m=float(rng.uniform(800.0, 1200.0)), height_m=500.0,
            sparsity=float(rng.uniform(0.02, 0.06)), snr_db=20.0,
            inner_steps=20, seed=1000 + i))
    return out


# --------------------------------------------------------------------------
# Geometry and scene draws
# --------------------------------------------------------------------------


def circular_track(n_pulses: int, radius_m: float, height_m: float,
                   span_deg: float, theta0_deg: float = 0.0) -> np.ndarray:
    """Platform positions gamma(s), shape (P, 3), float64."""
    if n_pulses == 1:
        theta = np.array([math.radians(theta0_deg)])
    else:
        theta = np.radians(theta0_deg) + np.radians(span_deg) * (
            np.arange(n_pulses, dtype=np.float64) / (n_pulses - 1))
    g = np.empty((n_pulses, 3), dtype=np.float64)
    g[:, 0] = radius_m * np.cos(theta)
    g[:, 1] = radius_m * np.sin(theta)
    g[:, 2] = height_m
    return g


def workload_track(w: Workload) -> np.ndarray:
    return circular_track(w.n_pulses, w.radius_m, w.height_m, w.span_deg,
                          w.theta0_deg)


def sampled_track(n_positions: int, radius_m: float, height_m: float,
                  span_deg: float, p: float, seed: int,
                  theta0_deg: float = 0.0) -> np.ndarray:
    """The pulses of the experiments' pulse selection: n_positions evenly
    spaced along the arc, each kept by its own Bernoulli(p) draw (the paper
    gives no p; it is an input here)."""
    full = circular_track(n_positions, radius_m, height_m, span_deg, theta0_deg)
    keep = np.random.default_rng(seed + 104729).random(n_positions) < p
    return full[keep]


def edgelet_atom_index(nx: int, ny: int, n_angles: int, length_idx: int,
                       angle_idx: int, x: int, y: int) -> int:
    """Atom number of the edgelet dictionary's documented order: (length,
    rotation, y, x) with x fastest."""
    return (length_idx * n_angles + angle_idx) * nx * ny + y * nx + x


def paper_scene(kind: str, nx: int, ny: int):
    """Coefficient vectors for scenes like the experiments' four (§IV-A:
    a square; two squares; lines of varying intensities, spaced; the same
    lines adjoined), rebuilt from the text (the images are not available):
    returns (lengths, angles_deg, c).  Squares use length-4 edgelets at 0 and
    90 degrees (4 atoms each), lines lengths 2, 4 and 6 at 0 degrees (5
    atoms).  An edgelet of length l covering columns xs .. xs + l - 1 is
    centred at xs + (l - 1) // 2."""
    n = nx * ny
    if kind in ("square", "two_squares"):
        lengths, angles = (4,), (0.0, 90.0)
        c = np.zeros(2 * n, dtype=np.complex128)
        corners = [(nx // 2 - 2, ny // 2 - 2)]
        if kind == "two_squares":
            corners = [(nx // 4 - 2, ny // 4 - 2), (3 * nx // 4 - 2, 3 * ny // 4 - 2)]
        for x0, y0 in corners:
            for (ai, x, y) in ((0, x0 + 1, y0), (0, x0 + 1, y0 + 3),
                               (1, x0, y0 + 1), (1, x0 + 3, y0 + 1)):
                c[edgelet_atom_index(nx, ny, 2, 0, ai, x, y)] = 1.0
        return lengths, angles, c
    if kind in ("lines_spaced", "lines_adjoined"):
        lengths, angles = (2, 4, 6), (0.0,)
        c = np.zeros(3 * n, dtype=np.complex128)
        # (length index, first column, row, intensity)
        if kind == "lines_spaced":
            lines = [(2, 2, 3, 1.0), (1, 12, 5, 0.8), (0, 20, 9, 0.6),
                     (2, 4, 15, 0.9), (1, 18, 21, 0.7)]
        else:  # end to end on two rows
            lines = [(2, 4, 10, 1.0), (1, 10, 10, 0.8), (0, 14, 10, 0.6),
                     (2, 6, 16, 0.9), (1, 12, 16, 0.7)]
        for li, xs, y, a in lines:
            l = lengths[li]
            c[edgelet_atom_index(nx, ny, 1, li, 0, xs + (l - 1) // 2, y)] = a
        return lengths, angles, c
    raise ValueError(kind)


def sparse_coefficients(m: int, frac: float, rng: np.random.Generator,
                        k: Optional[int] = None) -> np.ndarray:
    """k-sparse complex vector: |a| ~ U(0.5, 1), arg a ~ U[0, 2pi)."""
    if k is None:
        k = max(1, int(round(frac * m)))
    c = np.zeros(m, dtype=np.complex128)
    idx = rng.choice(m, size=k, replace=False)
    amp = rng.uniform(0.5, 1.0, size=k)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=k)
    c[idx] = amp * np.exp(1j * ph)
    return c


def clustered_coefficients(nx: int, ny: int, frac: float,
                           rng: np.random.Generator) -> np.ndarray:
    """3 x 3 pixel clusters around round(frac * N) centres, clipped at borders."""
    n = nx * ny
    k = max(1, int(round(frac * n)))
    centres = rng.choice(n, size=k, replace=False)
    img = np.zeros((ny, nx), dtype=np.complex128)
    for cidx in centres:
        i, j = divmod(int(cidx), nx)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                ii, jj = i + di, j + dj
                if 0 <= ii < ny and 0 <= jj < nx:
                    amp = rng.uniform(0.5, 1.0)
                    ph = rng.uniform(0.0, 2.0 * np.pi)
                    img[ii, jj] = amp * np.exp(1j * ph)
    return img.reshape(-1)


def workload_scene(w: Workload) -> np.ndarray:
    rng = np.random.default_rng(w.seed)
    if w.clustered:
        return clustered_coefficients(w.nx, w.ny, w.sparsity, rng)
    return sparse_coefficients(w.m_atoms, w.sparsity, rng)


def unit_noise(n_pulses: int, n_freq: int, seed: int) -> np.ndarray:
    """Unit-variance circular complex Gaussian draws, shape (P, K)."""
    rng = np.random.default_rng(seed + 7919)
    return (rng.standard_normal((n_pulses, n_freq))
            + 1j * rng.standard_normal((n_pulses, n_freq))) / np.sqrt(2.0)


def scale_noise(d_clean: np.ndarray, w: np.ndarray, snr_db: float) -> np.ndarray:
    """Per-pulse noise sigma_s w_s with sigma_s^2 = ||d_s||^2 / (K 10^(SNR/10))."""
    k = d_clean.shape[-1]
    p = np.sum(np.abs(d_clean) ** 2, axis=-1, keepdims=True)
    sigma = np.sqrt(p / (k * 10.0 ** (snr_db / 10.0)))
    return sigma * w


# --------------------------------------------------------------------------
# Philox4x32-10 and the Gaussian dictionary
# --------------------------------------------------------------------------

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: tuple) -> np.ndarray:
    """Philox4x32 with 10 rounds on a (..., 4) uint32 counter array."""
    x = [ctr[..., i].astype(np.uint64) for i in range(4)]
    k0 = np.uint64(key[0]) & _MASK32
    k1 = np.uint64(key[1]) & _MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + _PHILOX_W0) & _MASK32
            k1 = (k1 + _PHILOX_W1) & _MASK32
        p0 = _PHILOX_M0 * x[0]
        p1 = _PHILOX_M1 * x[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return np.stack([v.astype(np.uint32) for v in x], axis=-1)


def _u01_from_pair(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """53-bit uniform in (0, 1) from two 32-bit words: (k + 1/2) 2^-53."""
    v = (hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)
    return ((v >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian_dictionary_columns(n_pixels: int, cols: np.ndarray,
                                seed: int) -> np.ndarray:
    """Columns `cols` of the unit-norm complex Gaussian dictionary.

    Entry (n, j): Philox4x32-10 with counter (n, j, 0x5A5D1C7, 0) and key
    (seed mod 2^32, seed div 2^32); words (r0, r1) give u1, (r2, r3) give u2;
    z = sqrt(-2 ln u1) exp(2 pi i u2); each column is then divided by its
    2-norm.  Returns an (n_pixels, len(cols)) complex128 array.
    """
    cols = np.asarray(cols, dtype=np.int64)
    n = np.arange(n_pixels, dtype=np.uint64)
    ctr = np.zeros((n_pixels, cols.size, 4), dtype=np.uint32)
    ctr[..., 0] = n[:, None].astype(np.uint32)
    ctr[..., 1] = cols[None, :].astype(np.uint32)
    ctr[..., 2] = np.uint32(0x5A5D1C7)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    r = philox4x32_10(ctr, key)
    u1 = _u01_from_pair(r[..., 0], r[..., 1])
    u2 = _u01_from_pair(r[..., 2], r[..., 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    z = rad * (np.cos(2.0 * np.pi * u2) + 1j * np.sin(2.0 * np.pi * u2))
    z /= np.linalg.norm(z, axis=0, keepdims=True)
    return z


def gaussian_dictionary(n_pixels: int, n_atoms: int, seed: int,
                        chunk: int = 4096) -> np.ndarray:
    """Full N x M dictionary (Fortran order: each atom contiguous)."""
    d = np.empty((n_pixels, n_atoms), dtype=np.complex128, order="F")
    for j0 in range(0, n_atoms, chunk):
        j1 = min(n_atoms, j0 + chunk)
        d[:, j0:j1] = gaussian_dictionary_columns(
            n_pixels, np.arange(j0, j1), seed)
    return d


def workload_dictionary(w: Workload) -> Optional[np.ndarray]:
    """The random dictionary a workload draws (None for the pixel basis; the
    edgelet dictionary is no draw but part of the model, built by each side
    from its lengths and angles)."""
    if w.dictionary in ("identity", "edgelet"):
        return None
    return gaussian_dictionary(w.n_pixels, w.m_atoms, w.dict_seed)
