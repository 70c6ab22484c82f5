"""Helpers for the GPU parity tests: run the CUDA path and the FP64 oracle on
the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar
from tests.helpers import build_problem, oracle_config


def gpu_config(w, precision, lam=0.05, lambda_relative=True,
               power_iters_first=30, power_iters=4, margin=0.01,
               restart_momentum=False, compensated=True, host_dictionary=None,
               defer_gram=False):
    extra = {}
    if w.dictionary == "edgelet":
        dictionary, n_atoms = "edgelet", None
        extra = dict(edgelet_lengths=list(w.edgelet_lengths),
                     edgelet_angles=list(w.edgelet_angles))
    elif w.dictionary == "gaussian" and host_dictionary is None:
        dictionary, n_atoms = "gaussian", w.m_atoms
    elif host_dictionary is not None:
        dictionary, n_atoms = host_dictionary, host_dictionary.shape[1]
    else:
        dictionary, n_atoms = None, None
    return osar.make_config(
        w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz, pixel_m=w.pixel_m,
        precision=precision, dictionary=dictionary, n_atoms=n_atoms,
        dict_seed=w.dict_seed, lam=lam, lambda_relative=lambda_relative,
        power_iters_first=power_iters_first, power_iters=power_iters,
        lipschitz_margin=margin, restart_momentum=restart_momentum,
        compensated=compensated, defer_gram=defer_gram, **extra)


def run_pair(w, precision, steps, tol=0.0, pulses=None, lam=0.05,
             lambda_relative=True, restart_momentum=False, per_pulse=None,
             compensated=True, problem=None, host_dictionary=None,
             defer_gram=False):
    """Push the same pulses through the oracle and the GPU; call
    per_pulse(s, oracle, gpu) after each burst.  Returns (oracle, gpu)."""
    track, dic, c_true, data = problem if problem is not None else build_problem(w)
    P = track.shape[0] if pulses is None else pulses
    of = orc.OnlineFista(oracle_config(w, dic, lam=lam,
                                       lambda_relative=lambda_relative,
                                       restart_momentum=restart_momentum))
    gpu = osar.Osar(gpu_config(w, precision, lam=lam,
                               lambda_relative=lambda_relative,
                               restart_momentum=restart_momentum,
                               compensated=compensated,
                               host_dictionary=host_dictionary,
                               defer_gram=defer_gram))
    for s in range(P):
        of.push_pulse(track[s], data[s])
        gpu.push_pulse(track[s], data[s])
        n_o = of.iterate(steps, tol)
        n_g = gpu.iterate(steps, tol)
        if per_pulse is not None:
            per_pulse(s, of, gpu, n_o, n_g)
    return of, gpu
