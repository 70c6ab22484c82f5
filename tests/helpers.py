"""Shared test helpers: small seeded problems built from the input generator
and the FP64 oracle (the oracle supplies the clean measurements)."""
from __future__ import annotations

import numpy as np

from paper_2603_08582_gb300 import synth
from oracle import osar_oracle as orc


def small_workload(nx=8, ny=8, n_freq=16, n_pulses=16, span_deg=30.0,
                   dictionary="identity", n_atoms=None, sparsity=0.06,
                   snr_db=20.0, seed=0, f_lo=9.9e9, f_hi=10.1e9,
                   radius=1000.0, height=500.0, dict_seed=11,
                   edgelet_lengths=(), edgelet_angles=()):
    return synth.Workload(
        name=f"small_{nx}x{ny}_K{n_freq}_P{n_pulses}", nx=nx, ny=ny,
        n_freq=n_freq, f_lo_hz=f_lo, f_hi_hz=f_hi, n_pulses=n_pulses,
        span_deg=span_deg, radius_m=radius, height_m=height,
        dictionary=dictionary, n_atoms=n_atoms, dict_seed=dict_seed,
        sparsity=sparsity, snr_db=snr_db, seed=seed,
        edgelet_lengths=tuple(edgelet_lengths), edgelet_angles=tuple(edgelet_angles))


def workload_dictionary(w):
    """H for the oracle: the generator's draw, or the oracle's edgelets."""
    if w.dictionary == "edgelet":
        return orc.edgelet_dictionary(w.nx, w.ny, w.edgelet_lengths, w.edgelet_angles)
    return synth.workload_dictionary(w)


def build_problem(w, noise=True, c_true=None):
    """Track, dictionary, true coefficients and noisy data for workload w."""
    track = synth.workload_track(w)
    dictionary = workload_dictionary(w)
    if c_true is None:
        c_true = synth.workload_scene(w)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    clean = np.stack([
        orc.simulate_pulse(orc.forward_block(orc.phase_matrix(g, x, f),
                                             dictionary), c_true)
        for g in track])
    if noise:
        data = clean + synth.scale_noise(
            clean, synth.unit_noise(w.n_pulses, w.n_freq, w.seed), w.snr_db)
    else:
        data = clean
    return track, dictionary, c_true, data


def oracle_config(w, dictionary, lam=0.05, lambda_relative=True,
                  power_iters_first=30, power_iters=4, margin=0.01,
                  restart_momentum=False):
    return orc.OracleConfig(
        nx=w.nx, ny=w.ny, pixel_m=w.pixel_m, n_freq=w.n_freq,
        f_lo_hz=w.f_lo_hz, f_hi_hz=w.f_hi_hz, dictionary=dictionary,
        lam=lam, lambda_relative=lambda_relative,
        power_iters_first=power_iters_first, power_iters=power_iters,
        lipschitz_margin=margin, restart_momentum=restart_momentum)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    if den == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / den)


# Parity bars.  Every comparison with the oracle bounds the relative 2-norm
# error AND the worst element (relative to the largest reference entry), so a
# wrong small entry cannot hide under a small norm error.
def assert_close(got, ref, tol, what=""):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    e2 = rel_err(got, ref)
    assert e2 <= tol, f"{what}: relative 2-norm error {e2:.3e} > {tol:.1e}"
    if ref.size:
        scale = float(np.max(np.abs(ref)))
        einf = float(np.max(np.abs(got - ref)))
        bound = tol * scale if scale > 0 else tol
        assert einf <= bound, (f"{what}: worst element error {einf:.3e} > "
                               f"{tol:.1e} x max|ref| = {bound:.3e}")
    return e2


# Support comparison band: coefficient i may be zero on one side and non-zero
# on the other only when the oracle's last pre-shrink value satisfies
# ||u_i| - lambda tau| <= delta max|u|, with delta the precision's
# coefficient tolerance (a flip there is rounding, not a wrong step).
SUPPORT_DELTA = {"fp64": 1e-7, "fp32": 1e-4, "split_bf16": 1e-3}


def support_mismatch(c_got, state, delta):
    """Count of coefficients whose zero / non-zero status differs from the
    oracle state's c_hat away from the threshold band; also returns the
    number of coordinates inside the band."""
    c_got = np.asarray(c_got)
    if state.u is None or state.lip <= 0.0:
        diff = (np.abs(c_got) > 0) != (np.abs(state.c_hat) > 0)
        return int(np.count_nonzero(diff)), 0
    alpha = state.lam / state.lip
    mag = np.abs(state.u)
    near = np.abs(mag - alpha) <= delta * max(float(np.max(mag)), alpha)
    diff = (np.abs(c_got) > 0) != (np.abs(state.c_hat) > 0)
    return int(np.count_nonzero(diff & ~near)), int(np.count_nonzero(near))


def assert_coeffs(c_got, state, tol, delta, what="c"):
    """Coefficients against an oracle state: 2-norm, worst element, support."""
    e = assert_close(c_got, state.c_hat, tol, what)
    bad, _ = support_mismatch(c_got, state, delta)
    assert bad == 0, f"{what}: {bad} support differences outside the threshold band"
    return e


def host_gaussian_dictionary(n_pixels, n_atoms, seed, chunk=256, workers=None):
    """The input generator's Philox dictionary (synth.gaussian_dictionary),
    its column chunks drawn on a thread pool (NumPy releases the GIL inside
    its array operations); bitwise the generator's own columns."""
    import concurrent.futures as cf
    import os
    d = np.empty((n_pixels, n_atoms), dtype=np.complex128, order="F")

    def job(j0):
        j1 = min(n_atoms, j0 + chunk)
        d[:, j0:j1] = synth.gaussian_dictionary_columns(
            n_pixels, np.arange(j0, j1), seed)

    with cf.ThreadPoolExecutor(workers or os.cpu_count() or 1) as ex:
        list(ex.map(job, range(0, n_atoms, chunk)))
    return d


def dictionary_pulses(w, dictionary, pulses):
    """The first `pulses` pulses of workload w with a dense dictionary:
    d_s = F_s (H c_true) + noise at the workload's SNR (the clean part in the
    oracle's forward model, associated as F (H c))."""
    track = synth.workload_track(w)[:pulses]
    c_true = synth.workload_scene(w)
    rho = dictionary @ c_true
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    clean = np.stack([orc.phase_matrix(g, x, f) @ rho for g in track])
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)[:pulses]
    return track, c_true, clean + synth.scale_noise(clean, noise, w.snr_db)
