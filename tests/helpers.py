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
