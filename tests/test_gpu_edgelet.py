"""Edgelet dictionary (§III-A): binary atoms, so the forward block A_s = F_s H
is a sum of phase rows per atom on the GPU (no GEMM, no dictionary in device
memory).  Parity against the FP64 oracle, which builds H from its own
rasterisation (tests/test_oracle_pins.py pins it) and forms F_s H by a plain
matrix product: every pulse, the experiments' two dictionaries and a
diagonal one, ragged atom counts, all three precisions, the simulated data,
and the deferred Gram update.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config, run_pair

pytestmark = pytest.mark.gpu

TOL = {
    "fp64": {"gram": 1e-9, "b": 1e-9, "c": 1e-7},
    "fp32": {"gram": 2e-6, "b": 2e-6, "c": 1e-4},
    "split_bf16": {"gram": 1e-4, "b": 1e-4, "c": 1e-3},
}

DICTS = {
    # the experiments' dictionary for the square scenes: length 4, 0 and 90
    "squares": ((4,), (0.0, 90.0)),
    # the experiments' dictionary for the line scenes: lengths 2, 4, 6, 0 deg
    "lines": ((2, 4, 6), (0.0,)),
    # diagonals (a reading: steps of 45 degrees)
    "diagonal": ((3,), (45.0, 135.0)),
}


def _w(name, nx=12, ny=12, n_freq=40, n_pulses=5, seed=9):
    lengths, angles = DICTS[name]
    return small_workload(nx=nx, ny=ny, n_freq=n_freq, n_pulses=n_pulses,
                          dictionary="edgelet", edgelet_lengths=lengths,
                          edgelet_angles=angles, sparsity=0.02, seed=seed)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
@pytest.mark.parametrize("name", sorted(DICTS))
def test_edgelet_parity_every_pulse(prec, name):
    # 12 x 12 pixels: M = 288 / 432 / 288 atoms (3 or 4 blocks, ragged), K = 40
    w = _w(name)
    t = TOL[prec]

    def check(s, of, g, no, ng):
        assert_close(g.gram(), of.s.gram, t["gram"], "gram")
        assert_close(g.b(), of.s.b, t["b"], "b")
        assert_coeffs(g.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec])
        st = g.state()
        assert st["n"] == of.s.n
        assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10

    run_pair(w, prec, steps=10, per_pulse=check)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_edgelet_simulated_pulse_matches_the_oracle(prec):
    w = _w("lines", nx=10, ny=7, n_freq=24)
    track, dic, c_true, _ = build_problem(w)
    g = osar.Osar(gpu_config(w, prec))
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    for s in (0, 3):
        want = orc.simulate_pulse(orc.forward_block(orc.phase_matrix(track[s], x, f), dic),
                                  c_true)
        assert rel_err(g.simulate_pulse(track[s], c_true), want) <= 1e-9


def test_edgelet_larger_scene_and_deferred_update():
    # 32 x 32 pixels, the square dictionary: M = 2048 (16 blocks), K = 64
    w = _w("squares", nx=32, ny=32, n_freq=64, n_pulses=4, seed=12)
    of, g = run_pair(w, "split_bf16", steps=12)
    assert_coeffs(g.coeffs(), of.s, TOL["split_bf16"]["c"], SUPPORT_DELTA["split_bf16"])
    _, gd = run_pair(w, "split_bf16", steps=12, defer_gram=True)
    assert np.array_equal(g.gram(), gd.gram())
    assert_coeffs(gd.coeffs(), of.s, TOL["split_bf16"]["c"], SUPPORT_DELTA["split_bf16"])
