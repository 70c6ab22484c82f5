"""Deferred Gram update (defer_gram): pulse n's power steps and FISTA steps
apply G_n x as G_{n-1} x + A_n^H (A_n x) while the side stream forms G_n into
a second buffer.  The Gram is the update of Eq. 12 itself, so it must stay
bitwise the one of the in-order update; the iterates are G_n x in another
order of summation and must meet the split-BF16 parity bar against the FP64
oracle (Algorithm 1), and agree with the in-order run to rounding."""
import os

import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config, run_pair

pytestmark = pytest.mark.gpu

TOL_GRAM, TOL_B, TOL_C = 1e-4, 1e-4, 1e-3  # split-BF16 bar (test_gpu_parity)


def _ragged():
    # 24 x 24 pixels (N = 576), M = 1100 atoms (9 blocks, ragged), K = 96
    return small_workload(nx=24, ny=24, n_freq=96, n_pulses=8,
                          dictionary="gaussian", n_atoms=1100, sparsity=0.03,
                          seed=21, dict_seed=4)


def _small():
    # 12 x 12 pixels (N = 144), M = 300 atoms (3 blocks, ragged), K = 40
    return small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                          dictionary="gaussian", n_atoms=300, sparsity=0.03,
                          seed=5, dict_seed=77)


def _ctx(w, defer):
    return osar.Osar(gpu_config(w, "split_bf16", defer_gram=defer))


@pytest.mark.parametrize("make", [_small, _ragged])
def test_defer_matches_oracle_every_pulse(make):
    w = make()

    def check(s, of, g, no, ng):
        # the burst ran on G_{n-1} + the block's term; gram() then waits for G_n
        assert_close(g.b(), of.s.b, TOL_B, "b")
        assert_coeffs(g.coeffs(), of.s, TOL_C, SUPPORT_DELTA["split_bf16"])
        assert_close(g.gram(), of.s.gram, TOL_GRAM, "gram")
        st = g.state()
        assert st["n"] == of.s.n
        assert abs(st["lipschitz"] - of.s.lip) <= 1e-6 * of.s.lip * 10
        assert abs(st["t"] - of.s.t) <= 1e-9 * of.s.t

    run_pair(w, "split_bf16", steps=12, per_pulse=check, defer_gram=True)


def test_defer_gram_is_bitwise_the_in_order_update():
    w = _ragged()
    track, _, _, data = build_problem(w)
    a, b = _ctx(w, False), _ctx(w, True)
    for s in range(len(track)):
        for g in (a, b):
            g.push_pulse(track[s], data[s])
            g.iterate(12, 0.0, want_count=False)
    assert np.array_equal(a.gram(), b.gram())
    assert np.array_equal(a.b(), b.b())
    assert rel_err(b.coeffs(), a.coeffs()) <= 1e-4
    sa, sb = a.state(), b.state()
    assert sa["n"] == sb["n"] and sa["t"] == sb["t"]
    assert abs(sa["lipschitz"] - sb["lipschitz"]) <= 1e-5 * sa["lipschitz"]


def test_defer_stop_rule_host_waits_and_reads_mid_burst():
    w = _ragged()
    track, _, _, data = build_problem(w)
    ref, g = _ctx(w, False), _ctx(w, True)
    for s in range(len(track)):
        for x in (ref, g):
            x.push_pulse(track[s], data[s])
        if s == 2:
            # the Gram read mid-burst waits for G_n; the rest of the burst
            # uses it directly
            for x in (ref, g):
                x.iterate(3, 0.0, want_count=False)
            assert np.array_equal(ref.gram(), g.gram())
            for x in (ref, g):
                x.iterate(9, 0.0, want_count=False)
        else:
            na = ref.iterate(20, 1e-4)
            nb = g.iterate(20, 1e-4)
            assert abs(na - nb) <= 1
        if s % 3 == 1:
            g.synchronize()                      # main stream idle at the next push
    # the stop rule may end a burst one step apart: the split-BF16 bar
    assert rel_err(g.coeffs(), ref.coeffs()) <= TOL_C
    assert np.array_equal(ref.gram(), g.gram())


def test_defer_gram_apply_sees_the_pushed_pulse():
    w = _small()
    track, _, _, data = build_problem(w)
    ref, g = _ctx(w, False), _ctx(w, True)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms)
    for s in range(4):
        for c in (ref, g):
            c.push_pulse(track[s], data[s])
        # pushed, update pending: the apply waits for G_n
        assert rel_err(g.gram_apply(x), ref.gram_apply(x)) <= 1e-6
        for c in (ref, g):
            c.iterate(6, 0.0, want_count=False)


def test_defer_checkpoint_resume_is_bitwise(tmp_path):
    w = _ragged()
    track, _, _, data = build_problem(w)
    full = _ctx(w, True)
    part = _ctx(w, True)
    for s in range(4):
        for c in (full, part):
            c.push_pulse(track[s], data[s])
            c.iterate(10, 0.0, want_count=False)
    path = os.path.join(tmp_path, "ck.bin")
    part.save(path)                              # waits for the pending update
    part.close()
    resumed = osar.Osar.load(path, gpu_config(w, "split_bf16", defer_gram=True))
    for s in range(4, len(track)):
        for c in (full, resumed):
            c.push_pulse(track[s], data[s])
            c.iterate(10, 0.0, want_count=False)
    assert np.array_equal(full.coeffs(), resumed.coeffs())
    assert np.array_equal(full.gram(), resumed.gram())
    assert full.state() == resumed.state()
