"""The per-kernel timers (osar_profile_*): class selection and launch
sampling.  Instrumentation only, no paper counterpart: the bench's rooflines
divide algorithmic bytes by these times, so which launches they bracket has
to be exactly what the calls say.

* Selecting one class brackets that class's launches only.
* Sampling one launch in `every` brackets ceil(n / every) of the n launches
  a run with every launch bracketed sees (launch sequences are
  deterministic), and each sampled time is a real kernel time.
* Invalid masks, classes and strides are refused."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar, synth

pytestmark = pytest.mark.gpu


def _run(select=None, sample=None, pulses=3, steps=6):
    w = synth.Workload(name="profile_32x32", nx=32, ny=32, n_freq=128,
                       f_lo_hz=9.75e9, f_hi_hz=10.25e9, n_pulses=pulses,
                       span_deg=10.0, sparsity=0.05, snr_db=25.0, seed=3)
    cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                           precision="split_bf16")
    track = synth.workload_track(w)
    rng = np.random.default_rng(5)
    data = (rng.standard_normal((pulses, w.n_freq))
            + 1j * rng.standard_normal((pulses, w.n_freq)))
    with osar.Osar(cfg) as g:
        g.profile_reset()
        if select is not None:
            g.profile_select(*select)
        if sample is not None:
            g.profile_sample(*sample)
        g.profile_enable(True)
        for s in range(pulses):
            g.push_pulse(track[s], data[s])
            g.iterate(steps)
        out = {k: g.profile_read(k) for k in osar.KERNEL_CLASSES}
        g.profile_enable(False)
    return out


def test_select_brackets_only_the_chosen_class():
    full = _run()
    assert full["matvec"][0] > 0 and full["fista_finalize"][0] > 0
    only = _run(select=("matvec",))
    assert only["matvec"][0] == full["matvec"][0]
    for k, (n, ms) in only.items():
        if k != "matvec":
            assert n == 0 and ms == 0.0, k


@pytest.mark.parametrize("every", [2, 3, 5])
def test_sample_brackets_one_launch_in_every(every):
    full = _run()
    samp = _run(sample=("matvec", every))
    n = full["matvec"][0]
    assert samp["matvec"][0] == -(-n // every)
    assert samp["matvec"][1] > 0.0
    # the other classes keep every launch
    assert samp["fista_finalize"][0] == full["fista_finalize"][0]


def test_invalid_profile_arguments_are_refused():
    cfg = osar.make_config(32, 32, 128, 9.75e9, 10.25e9, precision="fp32")
    with osar.Osar(cfg) as g:
        lib, h = g._lib, g._h
        assert lib.osar_profile_select(h, 1 << len(osar.KERNEL_CLASSES)) == osar.OSAR_E_INVALID
        assert lib.osar_profile_sample(h, len(osar.KERNEL_CLASSES), 2) == osar.OSAR_E_INVALID
        assert lib.osar_profile_sample(h, -1, 2) == osar.OSAR_E_INVALID
        assert lib.osar_profile_sample(h, 4, 0) == osar.OSAR_E_INVALID
        # the context stays usable after a refused call
        g.profile_select("matvec")
        g.profile_sample("matvec", 1)
