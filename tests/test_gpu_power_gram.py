"""Power step fused into the Gram update (fuse_power_gram): the pair kernel's
epilogue holds each updated 128 x 128 block of G_n and applies it to the
power vector v, so the first power step of a pulse (Eq. 11) reads no Gram.

Pins: with one power step per pulse, L_n = max(L_{n-1}, (1 + margin) mu_n)
and v_n = G_n v_{n-1} / |G_n v_{n-1}| are formed on the host from the GPU's
own Gram (FP64, hi + compensation) and checked against the GPU's L_n every
pulse, so every block's row and column terms enter (v turns complex after
the first pulse, which also exposes a conjugation error).  Against separate
passes: the Gram and b stay bitwise, L_n and the coefficients agree to
rounding; against the FP64 oracle the split-BF16 bar holds; two runs give
the same bits."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config, run_pair

pytestmark = pytest.mark.gpu

TOL_GRAM, TOL_B, TOL_C = 1e-4, 1e-4, 1e-3  # split-BF16 bar (test_gpu_parity)


def _pixels():
    # 40 x 40 pixel basis: M = 1600, 13 blocks (a pair whose second block is
    # missing), K = 128
    return small_workload(nx=40, ny=40, n_freq=128, n_pulses=5, sparsity=0.03,
                          seed=32)


def _dictionary():
    # 24 x 24 pixels, M = 1100 Gaussian atoms (9 blocks, ragged), K = 96
    return small_workload(nx=24, ny=24, n_freq=96, n_pulses=5,
                          dictionary="gaussian", n_atoms=1100, sparsity=0.03,
                          seed=31, dict_seed=6)


def _ctx(w, fused, power_first=30, power=4):
    cfg = gpu_config(w, "split_bf16", power_iters_first=power_first,
                     power_iters=power)
    cfg.fuse_power_gram = 1 if fused else 0
    return osar.Osar(cfg)


@pytest.mark.parametrize("make", [_pixels, _dictionary])
def test_fused_power_step_matches_host_power_iteration(make):
    w = make()
    track, _, _, data = build_problem(w)
    g = _ctx(w, True, power_first=1, power=1)
    M = g.m_atoms
    v = np.full(M, 1.0 / np.sqrt(M), dtype=np.complex128)  # the initial vector
    lip = 0.0
    for s in range(len(track)):
        g.push_pulse(track[s], data[s])
        G = g.gram()
        y = G @ v
        mu = float(np.real(np.vdot(v, y)))
        lip = max(lip, 1.01 * mu)
        got = g.state()["lipschitz"]
        assert abs(got - lip) <= 1e-5 * lip, (s, got, lip)
        v = y / np.linalg.norm(y)
        if s >= 1:
            assert np.max(np.abs(v.imag)) > 1e-3 * np.max(np.abs(v.real))


@pytest.mark.parametrize("make", [_pixels, _dictionary])
def test_fused_power_step_against_separate_passes(make):
    w = make()
    track, _, _, data = build_problem(w)
    a, b = _ctx(w, False), _ctx(w, True)
    for s in range(len(track)):
        for g in (a, b):
            g.push_pulse(track[s], data[s])
            g.iterate(12, 0.0, want_count=False)
        sa, sb = a.state(), b.state()
        assert abs(sa["lipschitz"] - sb["lipschitz"]) <= 1e-5 * sa["lipschitz"]
    assert np.array_equal(a.gram(), b.gram())
    assert np.array_equal(a.b(), b.b())
    assert rel_err(b.coeffs(), a.coeffs()) <= 1e-4
    assert a.state()["t"] == b.state()["t"]


def test_fused_power_step_meets_the_oracle_bar():
    w = _dictionary()

    def check(s, of, g, no, ng):
        assert_close(g.b(), of.s.b, TOL_B, "b")
        assert_close(g.gram(), of.s.gram, TOL_GRAM, "gram")
        assert_coeffs(g.coeffs(), of.s, TOL_C, SUPPORT_DELTA["split_bf16"])
        assert abs(g.state()["lipschitz"] - of.s.lip) <= 1e-5 * of.s.lip

    run_pair(w, "split_bf16", steps=12, per_pulse=check)


def test_fused_power_step_is_deterministic():
    w = _pixels()
    track, _, _, data = build_problem(w)
    runs = []
    for _ in range(2):
        g = _ctx(w, True)
        for s in range(len(track)):
            g.push_pulse(track[s], data[s])
            g.iterate(10, 0.0, want_count=False)
        runs.append((g.coeffs(), g.state()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
