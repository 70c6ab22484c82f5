"""FP64 CPU oracle for Online FISTA (Flynn, Ivanov, Yazici, "Online Sparse
Synthetic Aperture Radar Imaging", arXiv 2603.08582).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  It shares no code with the CUDA library.

Everything here is plain NumPy in float64 / complex128, written in the
paper's order and notation, with no blocking, fusion or reordering beyond
what each definition states.  Library primitives (matmul, norm, exp) serve as
single steps.

Readings taken where the paper is silent, ambiguous or garbled:

* phase sign: F[m, n] = exp(-i 2 k_m R_n) with R_n = |gamma(s) - x_n| and
  k_m = 2 pi f_m / c (Eqs. 2-4; the sign is a convention, used for both
  simulation and inversion);
* frequencies f_m = linspace(f_lo, f_hi, K), both ends inclusive (the N_r
  fast-time samples of §II read as K frequency samples); amplitude A = 1;
* R_n = I (white noise), so Eq. 12 becomes dA = G^H G, db = G^H d, unless
  a pulse gives its K noise variances (R_n diagonal: frequencies with
  independent noise; a full covariance is not taken);
* the threshold of Algorithm 1 is S_{lambda tau} (the printed "t tau" is read
  as a typo) and the shrinkage is the complex one,
  S_a(u) = u max(0, 1 - a / |u|), which is 0 whenever |u| <= a;
* coefficients are complex (c in C^M);
* lambda_n = lambda_rel * ||b_n||_inf recomputed at every pulse (or an
  absolute lambda);
* L_n = max(L_{n-1}, (1 + delta_L) mu_n) where mu_n is the Rayleigh quotient
  of a warm-started power iteration on the accumulated Gram (Eq. 11); the
  increments are PSD so the largest eigenvalue never decreases;
* the momentum scalar t is carried across pulses and the vector z restarts at
  c_hat_{n-1} (Algorithm 1, initialisation); restart_momentum=True resets
  t = 1 at every pulse instead;
* an optional stop rule ends a burst once ||c^(k) - z^(k)||_2 <=
  tol ||c^(k)||_2 (tol = 0 means exactly m steps, as in the paper);
* edgelet atoms (§III-A) step by (round(cos psi), round(sin psi)) for psi
  a multiple of 45 degrees, cover j - (l - 1) // 2 steps from their centre
  (j = 0 .. l - 1), drop pixels off the grid, and run over (length,
  rotation, y, x) with x fastest;
* repeated bursts without a new pulse continue the same run of Algorithm 1
  (z, c^(k-1) and t are kept), so two bursts of a and b steps equal one burst
  of a + b steps.

* the SNR of Eq. 18 takes mu as an RMS amplitude (20 log10 of an amplitude
  ratio) and, since the scenes' images are not given, is read in the
  coefficient domain: the true atoms against the rest.

Parity status: every function below is pinned by closed forms, invariants,
brute force or an independent solver in tests/test_oracle_pins.py.  The
online trajectory has no closed form; `OnlineFista` is pinned pulse by pulse
instead: lambda_n against the batch data vector, L_n against G_n's spectrum
and the stored power vector, the warm start and the carried t, two bursts
equal to one, and every pulse's converged image against the LASSO optimality
conditions of that pulse's (G_n, b_n, lambda_n).  The noise draws are inputs
from the seeded generators, not part of this module.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

C_LIGHT = 299_792_458.0


# --------------------------------------------------------------------------
# Forward model (§II, Eqs. 1-4; §III-A, Eqs. 5-6)
# --------------------------------------------------------------------------


def pixel_positions(nx: int, ny: int, pixel_m: float) -> np.ndarray:
    """x_n = ((j - (nx-1)/2) dx, (i - (ny-1)/2) dx, 0), n = i nx + j (§II)."""
    i, j = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    x = np.zeros((ny * nx, 3), dtype=np.float64)
    x[:, 0] = ((j - (nx - 1) / 2.0) * pixel_m).reshape(-1)
    x[:, 1] = ((i - (ny - 1) / 2.0) * pixel_m).reshape(-1)
    return x


def frequencies(n_freq: int, f_lo: float, f_hi: float) -> np.ndarray:
    """f_m, m = 0..K-1, evenly spaced with both ends inclusive (§II)."""
    return np.linspace(f_lo, f_hi, n_freq)


def ranges(gamma: np.ndarray, x: np.ndarray) -> np.ndarray:
    """R_n = |gamma(s) - x_n| (Eq. 3)."""
    return np.sqrt(np.sum((np.asarray(gamma)[None, :] - x) ** 2, axis=1))


def phase_matrix(gamma: np.ndarray, x: np.ndarray,
                 freqs: np.ndarray) -> np.ndarray:
    """F[m, n] = exp(-i 2 k_m R_n), k_m = 2 pi f_m / c (Eqs. 2-4), K x N."""
    r = ranges(gamma, x)
    k = 2.0 * np.pi * freqs / C_LIGHT
    return np.exp(-1j * 2.0 * np.outer(k, r))


def edgelet_atoms(nx: int, ny: int, lengths, angles_deg) -> list:
    """Pixel sets of the edgelet dictionary (§III-A, Dictionary Model): each
    atom is a binary edgelet of length l and rotation psi centred at pixel
    (x, y), for every length, rotation and centre x < nx, y < ny.

    Readings (the paper gives no rasterisation): psi is a multiple of 45
    degrees and the edgelet steps by (round(cos psi), round(sin psi)) pixels;
    it covers the centre plus j - (l - 1) // 2 steps for j = 0 .. l - 1 (for
    even l one more pixel ahead of the centre than behind); pixels outside
    the grid are dropped; atoms run over (length, rotation, y, x) with x
    fastest; pixel (x, y) is index y * nx + x."""
    atoms = []
    for l in lengths:
        for a in angles_deg:
            dx = int(round(np.cos(np.radians(a))))
            dy = int(round(np.sin(np.radians(a))))
            for y in range(ny):
                for x in range(nx):
                    pix = []
                    for j in range(l):
                        o = j - (l - 1) // 2
                        px, py = x + o * dx, y + o * dy
                        if 0 <= px < nx and 0 <= py < ny:
                            pix.append(py * nx + px)
                    atoms.append(pix)
    return atoms


def edgelet_dictionary(nx: int, ny: int, lengths, angles_deg) -> np.ndarray:
    """The binary dictionary H (N x M, 1 on an atom's pixels, §III-A)."""
    atoms = edgelet_atoms(nx, ny, lengths, angles_deg)
    h = np.zeros((nx * ny, len(atoms)))
    for m, pix in enumerate(atoms):
        h[pix, m] = 1.0
    return h


def forward_block(f: np.ndarray, dictionary: Optional[np.ndarray]) -> np.ndarray:
    """Per-pulse forward operator G_n = F H (Eq. 6); H = I for a pixel basis."""
    if dictionary is None:
        return f
    return f @ dictionary


def simulate_pulse(a_s: np.ndarray, c_true: np.ndarray) -> np.ndarray:
    """Noise-free data d_n = G_n c (Eq. 5 without the noise term)."""
    return a_s @ c_true


# --------------------------------------------------------------------------
# Objective (§III-B, Eqs. 8-11)
# --------------------------------------------------------------------------


def gram_increment(a_s: np.ndarray, noise_var=None) -> np.ndarray:
    """dA_n = G_n^H R_n^{-1} G_n (Eq. 12); R_n = diag(noise_var), or I."""
    if noise_var is None:
        return a_s.conj().T @ a_s
    r_inv = np.diag(1.0 / np.asarray(noise_var, dtype=np.float64))
    return a_s.conj().T @ r_inv @ a_s


def data_increment(a_s: np.ndarray, d_s: np.ndarray, noise_var=None) -> np.ndarray:
    """db_n = G_n^H R_n^{-1} d_n (Eq. 12); R_n = diag(noise_var), or I."""
    if noise_var is None:
        return a_s.conj().T @ d_s
    r_inv = np.diag(1.0 / np.asarray(noise_var, dtype=np.float64))
    return a_s.conj().T @ r_inv @ d_s


def smooth_part(blocks, data, c) -> float:
    """f(c) = 1/2 sum_k |d_k - G_k c|^2 (Eq. 9, R_k = I)."""
    return 0.5 * sum(float(np.sum(np.abs(d - a @ c) ** 2))
                     for a, d in zip(blocks, data))


def lasso_objective(blocks, data, c, lam: float) -> float:
    """J_n(c) = f(c) + lambda ||c||_1 (Eq. 8), complex modulus in the l1 norm."""
    return smooth_part(blocks, data, c) + lam * float(np.sum(np.abs(c)))


def lasso_objective_gram(g: np.ndarray, b: np.ndarray, c: np.ndarray,
                         lam: float, const: float = 0.0) -> float:
    """Eq. 8 through the sufficient statistics: 1/2 c^H G c - Re(b^H c) + const
    + lambda ||c||_1, which equals J_n(c) when const = 1/2 sum |d_k|^2."""
    quad = 0.5 * float(np.real(np.vdot(c, g @ c)))
    lin = float(np.real(np.vdot(b, c)))
    return quad - lin + const + lam * float(np.sum(np.abs(c)))


def gradient_matrix_free(blocks, data, c) -> np.ndarray:
    """grad f(c) = sum_k G_k^H (G_k c - d_k) (Eq. 10), without a stored Gram."""
    out = np.zeros(blocks[0].shape[1], dtype=np.complex128)
    for a, d in zip(blocks, data):
        out += a.conj().T @ (a @ c - d)
    return out


def batch_gram(blocks) -> np.ndarray:
    """sum_k G_k^H G_k from the stacked operator [G_1; ...; G_n] (Eqs. 11-13),
    a different loop nest from the pulse-by-pulse recursion."""
    stacked = np.concatenate(blocks, axis=0)
    return stacked.conj().T @ stacked


def batch_data(blocks, data) -> np.ndarray:
    stacked = np.concatenate(blocks, axis=0)
    return stacked.conj().T @ np.concatenate(data)


def incremental_lipschitz_bound(l_prev: float, a_s: np.ndarray) -> float:
    """Eq. 14 read with the index slip removed: L_n <= L_{n-1} + ||G_n||_2^2."""
    return l_prev + float(np.linalg.norm(a_s, 2) ** 2)


# --------------------------------------------------------------------------
# Algorithm 1 building blocks
# --------------------------------------------------------------------------


def soft_threshold(u: np.ndarray, alpha: float) -> np.ndarray:
    """Complex shrinkage S_alpha(u) = u max(0, 1 - alpha/|u|) (Algorithm 1)."""
    u = np.asarray(u, dtype=np.complex128)
    mag = np.abs(u)
    out = np.zeros_like(u)
    keep = mag > alpha
    out[keep] = u[keep] * (1.0 - alpha / mag[keep])
    return out


def momentum_next(t: float) -> float:
    """t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 (Algorithm 1)."""
    return (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0


def power_iteration(g: np.ndarray, v: np.ndarray, steps: int):
    """Warm-started power iteration for the spectral norm of Eq. 11.

    Each step: w = G v, mu = Re(v^H w) with |v| = 1, v <- w / |w|.
    Returns (mu of the last step, the updated unit vector v).
    """
    v = v / np.linalg.norm(v)
    mu = 0.0
    for _ in range(steps):
        w = g @ v
        mu = float(np.real(np.vdot(v, w)))
        nw = np.linalg.norm(w)
        if nw == 0.0:
            break
        v = w / nw
    return mu, v


def kkt_residual(g: np.ndarray, b: np.ndarray, c: np.ndarray,
                 lam: float) -> float:
    """Max violation of the LASSO optimality conditions for Eq. 8.

    With grad = G c - b: on the support grad_i + lambda c_i/|c_i| = 0,
    off the support |grad_i| <= lambda.  Returned relative to lambda.
    """
    grad = g @ c - b
    mag = np.abs(c)
    on = mag > 0
    r_on = np.abs(grad[on] + lam * c[on] / mag[on])
    r_off = np.maximum(0.0, np.abs(grad[~on]) - lam)
    worst = 0.0
    if r_on.size:
        worst = max(worst, float(np.max(r_on)))
    if r_off.size:
        worst = max(worst, float(np.max(r_off)))
    return worst / lam


def fista_fixed(g: np.ndarray, b: np.ndarray, lam: float, lip: float,
                steps: int, c0: Optional[np.ndarray] = None,
                t1: float = 1.0):
    """Plain FISTA on a fixed (G, b) with tau = 1/L (Algorithm 1's inner loop
    with A_n, b_n held fixed).  Returns (c, t, list of iterates)."""
    tau = 1.0 / lip
    c_prev = np.zeros_like(b) if c0 is None else np.array(c0, dtype=np.complex128)
    z = c_prev.copy()
    t = t1
    hist = []
    for _ in range(steps):
        grad = g @ z - b
        u = z - tau * grad
        c = soft_threshold(u, lam * tau)
        t_next = momentum_next(t)
        z = c + ((t - 1.0) / t_next) * (c - c_prev)
        c_prev = c
        t = t_next
        hist.append(c)
    return c_prev, t, hist


def large_coefficient_count(c: np.ndarray, threshold: float = 2e-2) -> int:
    """Number of "large" coefficients, |c_m| > threshold (§IV-B counts them
    with threshold 2e-2 against slow time)."""
    return int(np.count_nonzero(np.abs(np.asarray(c)) > threshold))


def coefficient_snr_db(c: np.ndarray, support) -> float:
    """SNR of Eq. 18, 20 log10(mu_signal / mu_noise), with mu read as the RMS
    amplitude of the coefficients over the reference support (signal) and
    over the remaining coefficients (noise)."""
    mag = np.abs(np.asarray(c))
    on = np.zeros(mag.size, dtype=bool)
    on[np.asarray(support, dtype=np.int64)] = True
    mu_s = np.sqrt(np.mean(mag[on] ** 2))
    mu_n = np.sqrt(np.mean(mag[~on] ** 2)) if np.any(~on) else 0.0
    if mu_n == 0.0:
        return float("inf") if mu_s > 0 else float("nan")
    return float(20.0 * np.log10(mu_s / mu_n))


def memory_values(m_atoms: int, n_pixels: int, n_r: int, n: int):
    """Values stored (Table I): (FISTA, Online FISTA)."""
    fista = m_atoms * (n_pixels + 1) + (2 * n * n_r) * (1 + m_atoms + n_r)
    online = m_atoms * (n_pixels + 1) + (2 * m_atoms) * (m_atoms + 1)
    return fista, online


# --------------------------------------------------------------------------
# Online FISTA (§III-C, Eqs. 12-13, Algorithm 1)
# --------------------------------------------------------------------------


@dataclass
class OracleConfig:
    nx: int
    ny: int
    pixel_m: float
    n_freq: int
    f_lo_hz: float
    f_hi_hz: float
    dictionary: Optional[np.ndarray] = None      # N x M, None => identity
    lam: float = 0.05                             # lambda_rel or absolute
    lambda_relative: bool = True
    power_iters_first: int = 30
    power_iters: int = 4
    lipschitz_margin: float = 0.01
    restart_momentum: bool = False


@dataclass
class OnlineState:
    n: int = 0
    gram: Optional[np.ndarray] = None
    b: Optional[np.ndarray] = None
    c_hat: Optional[np.ndarray] = None
    t: float = 1.0
    lip: float = 0.0
    lam: float = 0.0
    v: Optional[np.ndarray] = None
    # inner-loop state of the current burst
    z: Optional[np.ndarray] = None
    c_prev: Optional[np.ndarray] = None
    fresh: bool = True
    converged: bool = False
    # u^(k) of the last step taken: kept so that a comparison can tell which
    # coefficients sat within rounding of the threshold |u_i| = lambda tau
    u: Optional[np.ndarray] = None
    history: list = field(default_factory=list)


class MatrixFreeGram:
    """The accumulated Gram A_n kept as its pulses' blocks: A_n x is applied as
    sum_k G_k^H R_k^{-1} (G_k x) (Eqs. 10, 12-13) without forming the M x M
    matrix, for problems whose Gram does not fit in host memory.  Supports
    `gram @ x`, so Algorithm 1 and the power iteration use it unchanged."""

    def __init__(self):
        self.blocks = []   # G_k (K x M)
        self.weights = []  # diagonal of R_k^{-1} (K), or None for R_k = I

    def add(self, a_s: np.ndarray, noise_var=None) -> None:
        self.blocks.append(a_s)
        self.weights.append(None if noise_var is None else
                            1.0 / np.asarray(noise_var, dtype=np.float64))

    def __matmul__(self, x: np.ndarray) -> np.ndarray:
        out = np.zeros(self.blocks[0].shape[1], dtype=np.complex128)
        for a, w in zip(self.blocks, self.weights):
            r = a @ x
            if w is not None:
                r = w * r
            out += (r.conj() @ a).conj()         # G_k^H r, without a copy of G_k^H
        return out

    def entries(self, rows, cols) -> np.ndarray:
        """A_n[rows[q], cols[q]] = sum_k conj(G_k[:, i]) R_k^{-1} G_k[:, j]."""
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        out = np.zeros(rows.size, dtype=np.complex128)
        for a, w in zip(self.blocks, self.weights):
            wa = a[:, cols] if w is None else w[:, None] * a[:, cols]
            out += np.sum(a[:, rows].conj() * wa, axis=0)
        return out


class OnlineFista:
    """Pulse-by-pulse reference: push_pulse applies Eqs. 12-13 and the L / lambda
    updates, iterate runs Algorithm 1's inner loop.  matrix_free=True keeps
    the Gram as a MatrixFreeGram (the same arithmetic by Eq. 10, for sizes
    whose M x M matrix does not fit in host memory)."""

    def __init__(self, cfg: OracleConfig, matrix_free: bool = False):
        self.cfg = cfg
        self.x = pixel_positions(cfg.nx, cfg.ny, cfg.pixel_m)
        self.f = frequencies(cfg.n_freq, cfg.f_lo_hz, cfg.f_hi_hz)
        m = self.x.shape[0] if cfg.dictionary is None else cfg.dictionary.shape[1]
        self.m = m
        self.matrix_free = matrix_free
        self.s = OnlineState(
            gram=MatrixFreeGram() if matrix_free else np.zeros((m, m), dtype=np.complex128),
            b=np.zeros(m, dtype=np.complex128),
            c_hat=np.zeros(m, dtype=np.complex128),
            v=np.full(m, 1.0 / np.sqrt(m), dtype=np.complex128))

    # --- per-pulse statistics -------------------------------------------
    def block(self, gamma) -> np.ndarray:
        return forward_block(phase_matrix(gamma, self.x, self.f),
                             self.cfg.dictionary)

    def push_pulse(self, gamma, d_s, noise_var=None) -> None:
        """One pulse; noise_var: the K variances of a non-white pulse
        (R_n = diag(noise_var)), None for R_n = I."""
        s, cfg = self.s, self.cfg
        a_s = self.block(gamma)
        if self.matrix_free:
            s.gram.add(a_s, noise_var)                           # Eq. 13, kept as blocks
        else:
            s.gram = s.gram + gram_increment(a_s, noise_var)     # Eq. 13
        s.b = s.b + data_increment(a_s, d_s, noise_var)          # Eq. 13
        s.n += 1
        if cfg.lambda_relative:
            s.lam = cfg.lam * float(np.max(np.abs(s.b)))
        else:
            s.lam = cfg.lam
        steps = cfg.power_iters_first if s.n == 1 else cfg.power_iters
        mu, s.v = power_iteration(s.gram, s.v, steps)
        s.lip = max(s.lip, (1.0 + cfg.lipschitz_margin) * mu)
        # Algorithm 1 initialisation for the next burst
        s.fresh = True
        s.converged = False

    # --- Algorithm 1 inner loop -----------------------------------------
    def iterate(self, steps: int, tol: float = 0.0) -> int:
        s, cfg = self.s, self.cfg
        if s.n == 0:
            raise RuntimeError("iterate before the first pulse")
        if s.fresh:
            s.c_prev = s.c_hat.copy()                    # c^(0) = c_hat_{n-1}
            s.z = s.c_prev.copy()                        # z^(1) = c^(0)
            if s.n == 1 or cfg.restart_momentum:
                s.t = 1.0                                # t_1 = 1
            s.fresh = False
        if s.converged:
            return 0
        tau = 1.0 / s.lip
        done = 0
        for _ in range(steps):
            grad = s.gram @ s.z - s.b                    # g^(k)
            u = s.z - tau * grad                         # u^(k)
            c = soft_threshold(u, s.lam * tau)           # c^(k)
            t_next = momentum_next(s.t)                  # t_{k+1}
            z_next = c + ((s.t - 1.0) / t_next) * (c - s.c_prev)
            stop = False
            if tol > 0.0:
                cn = np.linalg.norm(c)
                stop = np.linalg.norm(c - s.z) <= tol * cn
            s.c_prev, s.z, s.t, s.u = c, z_next, t_next, u
            done += 1
            if stop:
                s.converged = True
                break
        s.c_hat = s.c_prev.copy()                        # c_hat_n = c^(m)
        return done

    def snapshot(self) -> OnlineState:
        return copy.deepcopy(self.s)


def run_online(cfg: OracleConfig, track: np.ndarray, data: np.ndarray,
               steps: int, tol: float = 0.0, keep_history: bool = False):
    """Push every pulse of `track` / `data` and run a burst after each one."""
    of = OnlineFista(cfg)
    iters = []
    for s_idx in range(track.shape[0]):
        of.push_pulse(track[s_idx], data[s_idx])
        iters.append(of.iterate(steps, tol))
        if keep_history:
            of.s.history.append((of.s.c_hat.copy(), of.s.t, of.s.lip, of.s.lam))
    return of, iters
