"""Fused first step: the last power step of a push also applies the Gram to
the next burst's z_1 = c_hat, and the burst's first FISTA step uses that
pass.  Every result must be bitwise the one of separate passes, including
when the first iterate after a push runs no step, when a pulse is pushed
without a burst, around a checkpoint taken between push and iterate, with
the stop rule, and in both working precisions and the FP64 path."""
import os

import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _ctx(w, prec, fused):
    cfg = gpu_config(w, prec)
    cfg.fuse_first_step = 1 if fused else 0
    return osar.Osar(cfg)


def _same(a, b):
    assert np.array_equal(a.coeffs(), b.coeffs())
    assert a.state() == b.state()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fp64"])
def test_fused_first_step_is_bitwise_neutral(prec):
    w = small_workload(nx=20, ny=20, n_freq=64, n_pulses=6, sparsity=0.05,
                       seed=41)
    track, _, _, data = build_problem(w)
    a, b = _ctx(w, prec, False), _ctx(w, prec, True)
    for s in range(len(track)):
        counts = []
        for g in (a, b):
            g.push_pulse(track[s], data[s])
            if s == 2:
                g.iterate(0)                 # no step yet: the pass waits
            if s == 3:
                continue                     # a pulse without a burst
            counts.append(g.iterate(8, 1e-6 if s == 4 else 0.0))
        if counts:
            assert counts[0] == counts[1]
        _same(a, b)


def test_fused_first_step_across_a_checkpoint(tmp_path):
    w = small_workload(nx=16, ny=16, n_freq=48, n_pulses=4, dictionary="gaussian",
                       n_atoms=300, sparsity=0.04, seed=42, dict_seed=3)
    track, _, _, data = build_problem(w)
    ref = _ctx(w, "split_bf16", False)
    g = _ctx(w, "split_bf16", True)
    for s in range(3):
        for x in (ref, g):
            x.push_pulse(track[s], data[s])
    path = os.path.join(tmp_path, "ck.bin")
    g.save(path)                             # pushed, burst not started
    cfg = gpu_config(w, "split_bf16")
    h = osar.Osar.load(path, cfg)
    for x in (ref, g, h):
        x.iterate(10)
    _same(ref, g)
    _same(ref, h)
