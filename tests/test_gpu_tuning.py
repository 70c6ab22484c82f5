"""Online lambda tuning (paper_2603_08582_gb300.tuning) on the device: the
gradient of each update is the library's adjoint through the pulse's burst
(osar_unroll_grad); started from a lambda factor that over-shrinks, the
tuner lowers it, and the tuned run ends closer to the reference scene than
the untuned one.  osar_set_lambda itself: the next pulse's lambda_n uses the
new factor, and bad arguments are refused."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from paper_2603_08582_gb300.tuning import OnlineLambdaTuner
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _err(c, ref):
    return np.linalg.norm(c - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_tuner_lowers_an_over_shrinking_lambda(prec):
    w = small_workload(nx=16, ny=16, n_freq=48, n_pulses=24, sparsity=0.05,
                       snr_db=30.0, seed=31)
    track, _, c_true, data = build_problem(w)
    rho0 = 0.4
    plain = osar.Osar(gpu_config(w, prec, lam=rho0))
    tuned = osar.Osar(gpu_config(w, prec, lam=rho0))
    tuner = OnlineLambdaTuner(tuned, c_true, rho=rho0, steps=10, every=2, eta=0.3)
    for s in range(w.n_pulses):
        plain.push_pulse(track[s], data[s])
        tuned.push_pulse(track[s], data[s])
        tuner.after_push(s)
        plain.iterate(10)
        tuned.iterate(10)
    assert len(tuner.history) == w.n_pulses // 2
    assert tuner.rho < 0.5 * rho0
    assert all(h["d_lambda"] > 0 for h in tuner.history[:3])
    assert _err(tuned.coeffs(), c_true) < 0.8 * _err(plain.coeffs(), c_true)


def test_set_lambda_applies_from_the_next_pulse():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=3, seed=5)
    track, _, _, data = build_problem(w)
    g = osar.Osar(gpu_config(w, "fp64", lam=0.05))
    g.push_pulse(track[0], data[0])
    lam0 = g.state()["lambda"]
    g.set_lambda(0.1)
    assert g.state()["lambda"] == lam0          # the current pulse keeps it
    g.iterate(3)
    g.push_pulse(track[1], data[1])
    bmax = np.max(np.abs(g.b()))
    assert g.state()["lambda"] == pytest.approx(0.1 * bmax, rel=1e-12)
    for bad in ((-0.1, 0), (np.nan, 0), (0.1, 1), (0.1, -1)):
        with pytest.raises(osar.OsarError) as e:
            g.set_lambda(bad[0], l=bad[1])
        assert e.value.status == osar.OSAR_E_INVALID
