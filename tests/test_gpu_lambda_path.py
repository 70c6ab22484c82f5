"""Lambda path: several solutions of the same pulses that differ only in
lambda share one Gram, data vector, L_n and power iteration, and each Gram
pass serves two solutions.  Solution l must be bitwise the one a context
with lambda = lambdas[l] computes, match the FP64 oracle run with that
lambda, stop on its own under the tolerance rule, and survive a checkpoint."""
import os

import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, oracle_config, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

LAMS = [0.02, 0.05, 0.11]
TOL_C = {"fp64": 1e-7, "fp32": 1e-4, "split_bf16": 1e-3}


def _path_cfg(w, prec, lams):
    cfg = gpu_config(w, prec)
    lv = np.asarray(lams, dtype=np.float64)
    cfg.n_lambdas = len(lams)
    cfg.lambda_list = lv.ctypes.data
    cfg._keep_lams = lv
    return cfg


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fp64"])
def test_path_solutions_equal_single_contexts_and_oracles(prec):
    w = small_workload(nx=20, ny=20, n_freq=64, n_pulses=6, sparsity=0.05,
                       seed=51)
    track, dic, _, data = build_problem(w)
    path = osar.Osar(_path_cfg(w, prec, LAMS))
    singles = [osar.Osar(gpu_config(w, prec, lam=lam)) for lam in LAMS]
    oracles = [orc.OnlineFista(oracle_config(w, dic, lam=lam)) for lam in LAMS]
    for s in range(len(track)):
        path.push_pulse(track[s], data[s])
        path.iterate(12)
        for g, o in zip(singles, oracles):
            g.push_pulse(track[s], data[s])
            g.iterate(12)
            o.push_pulse(track[s], data[s])
            o.iterate(12)
        for l, (g, o) in enumerate(zip(singles, oracles)):
            st = path.lambda_state(l)
            assert np.array_equal(st["coeffs"], g.coeffs()), (prec, s, l)
            assert st["lambda"] == g.state()["lambda"]
            assert st["t"] == g.state()["t"]
            assert_coeffs(st["coeffs"], o.s, TOL_C[prec], SUPPORT_DELTA[prec],
                          f"c {prec} pulse {s} lambda {l}")
    assert np.array_equal(path.coeffs(), singles[0].coeffs())


def test_path_solutions_stop_on_their_own():
    w = small_workload(nx=16, ny=16, n_freq=48, n_pulses=4, sparsity=0.05,
                       seed=52)
    track, _, _, data = build_problem(w)
    lams = [0.01, 0.05, 0.2, 0.4]
    path = osar.Osar(_path_cfg(w, "fp64", lams))
    singles = [osar.Osar(gpu_config(w, "fp64", lam=lam)) for lam in lams]
    for s in range(len(track)):
        path.push_pulse(track[s], data[s])
        path.iterate(300, 1e-6)
        counts = []
        for l, g in enumerate(singles):
            g.push_pulse(track[s], data[s])
            counts.append(g.iterate(300, 1e-6))
            st = path.lambda_state(l)
            assert st["iters"] == counts[-1]
            assert np.array_equal(st["coeffs"], g.coeffs())
    assert len(set(counts)) > 1  # the solutions did stop at different steps


def test_path_checkpoint_resume(tmp_path):
    w = small_workload(nx=16, ny=16, n_freq=48, n_pulses=5, dictionary="gaussian",
                       n_atoms=300, sparsity=0.04, seed=53, dict_seed=5)
    track, _, _, data = build_problem(w)
    a = osar.Osar(_path_cfg(w, "split_bf16", LAMS))
    for s in range(3):
        a.push_pulse(track[s], data[s])
        a.iterate(8)
    path = os.path.join(tmp_path, "path.ck")
    a.save(path)
    b = osar.Osar.load(path, _path_cfg(w, "split_bf16", LAMS))
    for s in range(3, 5):
        for x in (a, b):
            x.push_pulse(track[s], data[s])
            x.iterate(8)
    for l in range(len(LAMS)):
        assert np.array_equal(a.lambda_state(l)["coeffs"], b.lambda_state(l)["coeffs"])
