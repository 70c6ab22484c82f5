"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative 2-norm unless stated):
  FP64 path       Gram, b  <= 1e-9   (phase reductions agree to ~1e-10 rad)
                  c        <= 1e-7   (required: 1e-5)
  FP32 path       Gram     <= 2e-6,  c <= 1e-4
  split-BF16      Gram     <= 1e-4   (bf16 hi+lo keeps 2^-17 per factor),
                  c        <= 1e-3   (required: 1e-3)
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar, synth
from tests.helpers import (small_workload, build_problem, oracle_config, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import run_pair, gpu_config

pytestmark = pytest.mark.gpu

TOL = {
    "fp64": {"gram": 1e-9, "b": 1e-9, "c": 1e-7},
    "fp32": {"gram": 2e-6, "b": 2e-6, "c": 1e-4},
    "split_bf16": {"gram": 1e-4, "b": 1e-4, "c": 1e-3},
}


def _check_state(prec, of, gpu, with_gram=True):
    """Gram, b, lambda_n, L_n, t and c against the oracle: relative 2-norm and
    worst element for the arrays, and the support of c away from the
    threshold band."""
    t = TOL[prec]
    if with_gram:
        assert_close(gpu.gram(), of.s.gram, t["gram"], "gram")
    assert_close(gpu.b(), of.s.b, t["b"], "b")
    st = gpu.state()
    assert st["n"] == of.s.n
    assert abs(st["lambda"] - of.s.lam) <= t["b"] * max(1.0, of.s.lam) * 10
    assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10
    assert abs(st["t"] - of.s.t) <= 1e-9 * of.s.t
    assert_coeffs(gpu.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_pixel_basis_small_every_pulse(prec):
    """16 x 16 pixels (2 Gram blocks), 24 frequencies (ragged), 10 pulses."""
    w = small_workload(nx=16, ny=16, n_freq=24, n_pulses=10, span_deg=25.0,
                       sparsity=0.05, seed=21)
    run_pair(w, prec, steps=12,
             per_pulse=lambda s, of, g, no, ng: _check_state(prec, of, g))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_gaussian_dictionary_ragged(prec):
    """12 x 12 pixels (N = 144), M = 300 atoms (3 blocks, ragged), K = 40."""
    w = small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                       dictionary="gaussian", n_atoms=300, sparsity=0.03,
                       seed=5, dict_seed=77)
    run_pair(w, prec, steps=10,
             per_pulse=lambda s, of, g, no, ng: _check_state(prec, of, g))


def test_host_dictionary_equals_device_gaussian():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=4,
                       dictionary="gaussian", n_atoms=130, dict_seed=9)
    problem = build_problem(w)
    d_host = synth.gaussian_dictionary(w.n_pixels, w.m_atoms, w.dict_seed)
    _, g1 = run_pair(w, "fp64", steps=8, problem=problem)
    _, g2 = run_pair(w, "fp64", steps=8, problem=problem, host_dictionary=d_host)
    assert rel_err(g1.gram(), g2.gram()) < 1e-12
    assert rel_err(g1.coeffs(), g2.coeffs()) < 1e-10


def test_c1_full_config_fp64():
    """The 32 x 32 pixel-basis workload at full size: 64 pulses, K = 128,
    20 warm-started steps per pulse; coefficients within 1e-5 of the oracle."""
    w = synth.workloads()["c1_32x32_fp64"]
    errs = []

    def check(s, of, g, no, ng):
        if s % 16 == 15 or s == w.n_pulses - 1:
            errs.append(rel_err(g.coeffs(), of.s.c_hat))

    of, gpu = run_pair(w, "fp64", steps=w.inner_steps, per_pulse=check)
    assert max(errs) <= 1e-7, errs
    assert_coeffs(gpu.coeffs(), of.s, 1e-7, SUPPORT_DELTA["fp64"])
    assert_close(gpu.gram(), of.s.gram, 1e-9, "gram")
    # point targets: the largest coefficients sit on true scatterers
    c_true = synth.workload_scene(w)
    top = np.argsort(-np.abs(gpu.coeffs()))[:10]
    assert np.all(np.abs(c_true[top]) > 0)


def test_c1_full_config_split_bf16_error_report():
    w = synth.workloads()["c1_32x32_fp64"]
    of, gpu = run_pair(w, "split_bf16", steps=w.inner_steps)
    eg = assert_close(gpu.gram(), of.s.gram, 1e-4, "gram")
    eb = assert_close(gpu.b(), of.s.b, 1e-4, "b")
    ec = assert_coeffs(gpu.coeffs(), of.s, 1e-3, SUPPORT_DELTA["split_bf16"])
    print(f"split-BF16 vs FP64 oracle on 32x32: gram {eg:.2e} b {eb:.2e} c {ec:.2e}")


def test_uncompensated_split_still_within_tolerance():
    w = small_workload(nx=16, ny=16, n_freq=32, n_pulses=8, seed=3)
    of, gpu = run_pair(w, "split_bf16", steps=10, compensated=False)
    assert_close(gpu.gram(), of.s.gram, 1e-4, "gram")
    assert_coeffs(gpu.coeffs(), of.s, 1e-3, SUPPORT_DELTA["split_bf16"])


def test_degenerate_single_pixel_single_frequency():
    w = small_workload(nx=1, ny=1, n_freq=1, n_pulses=3, sparsity=1.0, seed=2)
    run_pair(w, "fp64", steps=5,
             per_pulse=lambda s, of, g, no, ng: _check_state("fp64", of, g))


def test_absolute_lambda_restart_momentum_and_tolerance_stop():
    w = small_workload(nx=10, ny=10, n_freq=20, n_pulses=6, seed=8)
    counts = []

    def check(s, of, g, no, ng):
        counts.append((no, ng))
        _check_state("fp64", of, g)

    run_pair(w, "fp64", steps=300, tol=1e-5, lam=0.5, lambda_relative=False,
             restart_momentum=True, per_pulse=check)
    assert all(a == b for a, b in counts), counts
    assert any(a < 300 for a, _ in counts)


def test_iterate_split_equals_single_burst_and_state_rules():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=3, seed=4)
    track, dic, c_true, data = build_problem(w)
    a = osar.Osar(gpu_config(w, "fp64"))
    b = osar.Osar(gpu_config(w, "fp64"))
    with pytest.raises(osar.OsarError) as ei:
        a.iterate(3)
    assert ei.value.status == osar.OSAR_E_STATE
    for s in range(w.n_pulses):
        a.push_pulse(track[s], data[s])
        b.push_pulse(track[s], data[s])
        a.iterate(9)
        b.iterate(4)
        assert b.iterate(0) == 0
        b.iterate(5)
        assert np.array_equal(a.coeffs(), b.coeffs())
    with pytest.raises(osar.OsarError):
        a.push_pulse([np.nan, 0, 0], data[0])


def test_gram_apply_and_simulate_match_oracle():
    w = small_workload(nx=12, ny=12, n_freq=40, n_pulses=4,
                       dictionary="gaussian", n_atoms=300, dict_seed=5, seed=6)
    of, gpu = run_pair(w, "fp64", steps=3)
    x = synth.sparse_coefficients(w.m_atoms, 0.5, np.random.default_rng(1))
    assert_close(gpu.gram_apply(x), of.s.gram @ x, 1e-10, "gram apply")
    gamma = synth.workload_track(w)[2]
    c_true = synth.workload_scene(w)
    d_gpu = gpu.simulate_pulse(gamma, c_true)
    d_orc = orc.simulate_pulse(of.block(gamma), c_true)
    assert_close(d_gpu, d_orc, 1e-9, "simulated pulse")
    rows = np.array([0, 5, 299, 128, 17])
    cols = np.array([299, 5, 0, 7, 200])
    assert np.max(np.abs(gpu.gram_entries(rows, cols) - of.s.gram[rows, cols])) \
        <= 1e-9 * np.max(np.abs(of.s.gram))


def test_checkpoint_resume_is_bit_exact():
    w = small_workload(nx=16, ny=16, n_freq=24, n_pulses=6, seed=12)
    track, dic, c_true, data = build_problem(w)
    for prec in ("fp64", "split_bf16"):
        full = osar.Osar(gpu_config(w, prec))
        part = osar.Osar(gpu_config(w, prec))
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "ckpt.bin")
            for s in range(w.n_pulses):
                full.push_pulse(track[s], data[s])
                full.iterate(7)
                if s < 3:
                    part.push_pulse(track[s], data[s])
                    part.iterate(7)
                if s == 2:
                    part.save(path)
                    part.close()
                    part = osar.Osar.load(path, gpu_config(w, prec))
                if s >= 3:
                    part.push_pulse(track[s], data[s])
                    part.iterate(7)
        assert np.array_equal(full.coeffs(), part.coeffs())
        assert np.array_equal(full.gram(), part.gram())


def test_zero_data_keeps_zero_coefficients():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=3)
    track = synth.workload_track(w)
    gpu = osar.Osar(gpu_config(w, "split_bf16"))
    for s in range(3):
        gpu.push_pulse(track[s], np.zeros(w.n_freq, complex))
        gpu.iterate(5)
    assert np.all(gpu.coeffs() == 0)
    assert gpu.state()["lambda"] == 0.0


@pytest.mark.parametrize("defer", [False, True])
def test_full_size_128x128_sampled_entries_split_bf16(defer):
    """The 128 x 128 / M = 32768 workload in the bench's launch configuration
    (and with the deferred Gram update): Gram and data-vector entries on
    sampled atoms, and the matvec on sampled rows, against the FP64 oracle
    computed column by column."""
    w = synth.workloads()["c2_128x128_split_bf16"]
    track = synth.workload_track(w)
    rng = np.random.default_rng(0)
    P = 3
    data = (rng.standard_normal((P, w.n_freq)) + 1j * rng.standard_normal((P, w.n_freq)))
    gpu = osar.Osar(gpu_config(w, "split_bf16", defer_gram=defer))
    for s in range(P):
        gpu.push_pulse(track[s], data[s])
    gpu.iterate(2)
    cols = np.unique(np.concatenate([rng.choice(w.m_atoms, 40, replace=False),
                                     [0, 127, 128, w.m_atoms - 1]]))
    dcol = synth.gaussian_dictionary_columns(w.n_pixels, cols, w.dict_seed)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    g_ref = np.zeros((cols.size, cols.size), complex)
    b_ref = np.zeros(cols.size, complex)
    for s in range(P):
        a_s = orc.phase_matrix(track[s], x, f) @ dcol      # K x |cols|
        g_ref += a_s.conj().T @ a_s
        b_ref += a_s.conj().T @ data[s]
    rr, cc = np.meshgrid(np.arange(cols.size), np.arange(cols.size), indexing="ij")
    got = gpu.gram_entries(cols[rr.ravel()], cols[cc.ravel()]).reshape(cols.size, cols.size)
    scale = np.max(np.abs(np.diag(g_ref)))
    assert np.max(np.abs(got - g_ref)) <= 1e-4 * scale
    b_gpu = gpu.b()
    assert np.max(np.abs(b_gpu[cols] - b_ref)) <= 1e-4 * np.max(np.abs(b_ref))
    st = gpu.state()
    assert abs(st["lambda"] - 0.05 * np.max(np.abs(b_gpu))) <= 1e-12 * st["lambda"]
    # matvec on sampled rows with a vector supported on the sampled atoms
    xs = np.zeros(w.m_atoms, complex)
    xs[cols] = rng.standard_normal(cols.size) + 1j * rng.standard_normal(cols.size)
    y = gpu.gram_apply(xs)
    y_ref = g_ref @ xs[cols]
    assert np.max(np.abs(y[cols] - y_ref)) <= 1e-4 * np.max(np.abs(y_ref))
