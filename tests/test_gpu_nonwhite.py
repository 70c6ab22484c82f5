"""Non-white pulses (Eq. 12 with R_n = diag(noise variances)): the library
whitens the data and the rows of the pulse's phase block, so Gram, data
vector and iterates must match the FP64 oracle's literal G^H R^{-1} G and
G^H R^{-1} d every pulse, with white and non-white pulses mixed, for the
pixel basis, a Gaussian dictionary (overlapped synthesis; and the deferred
Gram update) and edgelets.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, oracle_config, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

TOL = {
    "fp64": {"gram": 1e-9, "b": 1e-9, "c": 1e-7},
    "fp32": {"gram": 2e-6, "b": 2e-6, "c": 1e-4},
    "split_bf16": {"gram": 1e-4, "b": 1e-4, "c": 1e-3},
}


def _run(w, prec, defer=False, steps=10):
    track, dic, _, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    g = osar.Osar(gpu_config(w, prec, defer_gram=defer))
    rng = np.random.default_rng(17)
    t = TOL[prec]
    for s in range(track.shape[0]):
        var = None if s % 3 == 2 else rng.uniform(0.3, 3.0, w.n_freq)
        of.push_pulse(track[s], data[s], var)
        g.push_pulse(track[s], data[s], var)
        of.iterate(steps)
        g.iterate(steps, want_count=False)
        assert_close(g.b(), of.s.b, t["b"], f"b {prec} pulse {s}")
        assert_coeffs(g.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec], f"c {prec} pulse {s}")
        assert_close(g.gram(), of.s.gram, t["gram"], f"gram {prec} pulse {s}")
        st = g.state()
        assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_non_white_pixel_basis(prec):
    _run(small_workload(nx=14, ny=10, n_freq=36, n_pulses=6, sparsity=0.05,
                        seed=23), prec)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_non_white_gaussian_dictionary(prec):
    _run(small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                        dictionary="gaussian", n_atoms=300, sparsity=0.03,
                        seed=5, dict_seed=77), prec)


def test_non_white_deferred_update_and_edgelets():
    _run(small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                        dictionary="gaussian", n_atoms=300, sparsity=0.03,
                        seed=5, dict_seed=77), "split_bf16", defer=True)
    _run(small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                        dictionary="edgelet", edgelet_lengths=(4,),
                        edgelet_angles=(0.0, 90.0), sparsity=0.02, seed=9),
         "split_bf16")


def test_non_white_rejects_bad_variances():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=1, seed=7)
    g = osar.Osar(gpu_config(w, "fp64"))
    track, _, _, data = build_problem(w)
    var = np.ones(w.n_freq)
    var[3] = 0.0
    with pytest.raises(osar.OsarError) as e:
        g.push_pulse(track[0], data[0], var)
    assert e.value.status == osar.OSAR_E_INVALID
    g.push_pulse(track[0], data[0], np.ones(w.n_freq))   # the context still works
    g.iterate(4)
