"""osar_get_metrics: the experiments' quality figures (§IV-B) computed on the
device, against the oracle's definitions.

* On a scene like the experiments' Scene 1 (a square of four length-4
  edgelets in a 32 x 32 grid, 4 km radius, 1 km altitude, 1000 positions
  over 2 degrees kept with p = 0.3, 20 dB, m = 20), pulse by pulse: the
  library's count and SNR of its own coefficients equal the oracle's
  functions applied to them, and track the oracle's own run; once the
  oracle's count reaches the ideal 4, the library's does too and its large
  coefficients are exactly the square's atoms.
* Edge cases: no support (SNR undefined), the whole index range as support,
  zero coefficients, out-of-range indices."""
import math

import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar, synth
from tests.helpers import oracle_config

pytestmark = pytest.mark.gpu

THR = 2e-2


def _scene1(prec):
    lengths, angles, c_true = synth.paper_scene("square", 32, 32)
    w = synth.Workload(name="paper_square_32x32", nx=32, ny=32, n_freq=128,
                       f_lo_hz=9.9e9, f_hi_hz=10.1e9, n_pulses=1000,
                       span_deg=2.0, radius_m=4000.0, height_m=1000.0,
                       dictionary="edgelet", edgelet_lengths=lengths,
                       edgelet_angles=angles, snr_db=20.0, seed=7)
    track = synth.sampled_track(1000, 4000.0, 1000.0, 2.0, 0.3, w.seed)
    dic = orc.edgelet_dictionary(32, 32, lengths, angles)
    x = orc.pixel_positions(32, 32, 1.0)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    clean = np.stack([orc.simulate_pulse(orc.forward_block(orc.phase_matrix(g, x, f), dic),
                                         c_true) for g in track])
    noise = synth.unit_noise(len(track), w.n_freq, w.seed)
    data = clean + synth.scale_noise(clean, noise, w.snr_db)
    cfg = osar.make_config(32, 32, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                           precision=prec, dictionary="edgelet",
                           edgelet_lengths=list(lengths),
                           edgelet_angles=list(angles), lam=0.05)
    return w, track, data, dic, c_true, cfg


def _near_threshold(c, band):
    return np.any(np.abs(np.abs(c) - THR) <= band)


@pytest.mark.parametrize("prec,band", [("fp64", 1e-9), ("split_bf16", 1e-4)])
def test_scene1_metrics_against_the_oracle(prec, band):
    w, track, data, dic, c_true, cfg = _scene1(prec)
    support = np.flatnonzero(c_true)
    of = orc.OnlineFista(oracle_config(w, dic))
    g = osar.Osar(cfg)
    reached = None
    for s in range(60):
        of.push_pulse(track[s], data[s])
        g.push_pulse(track[s], data[s])
        of.iterate(20)
        g.iterate(20)
        c = g.coeffs()
        m = g.metrics(THR, support)
        # the device reduction equals the definitions on the same vector
        assert m["n_large"] == orc.large_coefficient_count(c, THR)
        assert m["n_nonzero"] == int(np.count_nonzero(c))
        assert m["n_support"] == support.size
        assert m["large_outside_support"] == int(np.count_nonzero(
            np.abs(np.delete(c, support)) > THR))
        assert m["l1"] == pytest.approx(float(np.sum(np.abs(c))), rel=1e-12)
        assert m["max_abs"] == pytest.approx(float(np.max(np.abs(c))), rel=1e-15)
        snr = orc.coefficient_snr_db(c, support)
        if math.isfinite(snr):
            assert m["snr_db"] == pytest.approx(snr, rel=1e-10, abs=1e-10)
        else:
            assert m["snr_db"] == snr or (math.isnan(snr) and math.isnan(m["snr_db"]))
        # and the oracle's own run, away from the threshold
        n_orc = orc.large_coefficient_count(of.s.c_hat, THR)
        if not _near_threshold(of.s.c_hat, band):
            assert m["n_large"] == n_orc, (s, m["n_large"], n_orc)
        if n_orc == support.size and reached is None:
            reached = s + 1
            assert m["n_large"] == support.size
            assert m["large_outside_support"] == 0
            big = np.flatnonzero(np.abs(c) > THR)
            assert set(big) == set(support)
    assert reached is not None, "the oracle never reached the ideal count"
    print(f"{prec}: ideal count of 4 after {reached} pulses; "
          f"SNR {g.metrics(THR, support)['snr_db']:.1f} dB")


def test_metrics_edge_cases():
    w = synth.Workload(name="m", nx=8, ny=8, n_freq=16, f_lo_hz=9.9e9,
                       f_hi_hz=10.1e9, n_pulses=2, span_deg=10.0, seed=1)
    g = osar.Osar(osar.make_config(8, 8, 16, 9.9e9, 10.1e9, precision="fp32"))
    # before any pulse: c = 0
    m = g.metrics(THR)
    assert m["n_large"] == m["n_nonzero"] == 0 and m["l1"] == 0.0
    assert math.isnan(m["snr_db"])
    track = synth.workload_track(w)
    rng = np.random.default_rng(0)
    for s in range(2):
        g.push_pulse(track[s], rng.standard_normal(16) + 1j * rng.standard_normal(16))
        g.iterate(10)
    c = g.coeffs()
    m = g.metrics(0.0, np.arange(64))
    assert m["n_large"] == int(np.count_nonzero(c)) and m["rms_noise"] == 0.0
    assert m["snr_db"] == (math.inf if np.any(c != 0) else m["snr_db"])
    with pytest.raises(osar.OsarError) as e:
        g.metrics(THR, [0, 64])
    assert e.value.status == osar.OSAR_E_INVALID
    with pytest.raises(osar.OsarError) as e:
        g.metrics(-1.0)
    assert e.value.status == osar.OSAR_E_INVALID
    # the context is still usable
    assert g.metrics(THR, [3, 3, 5])["n_support"] == 2
