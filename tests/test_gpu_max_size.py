"""The largest contexts the configuration allows: 131072-row Grams (524800
packed blocks, 8.6e9 stored entries; about 105 GB on the device in
split-BF16), where every packed-block and entry index needs 64 bits.  One
pulse of 64 frequencies (Eqs. 12-13) and two FISTA steps; the Gram and the
data vector on sampled rows and columns against the FP64 oracle's
definitions computed column by column, and the matvec on sampled rows:

* a 512 x 256 pixel-basis scene (N = M = 131072);
* a 32 x 32 scene with 131072 Gaussian atoms (the dictionary's limit)."""
import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar, synth
from tests.helpers import assert_close
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _check(w, cols_dict):
    track = synth.workload_track(w)
    rng = np.random.default_rng(11)
    d = rng.standard_normal(w.n_freq) + 1j * rng.standard_normal(w.n_freq)
    g = osar.Osar(gpu_config(w, "split_bf16"))
    g.push_pulse(track[0], d)
    assert g.iterate(2) == 2
    m = w.m_atoms
    cols = np.unique(np.concatenate([rng.choice(m, 36, replace=False),
                                     [0, 127, 128, m // 2, m - 129, m - 128, m - 1]]))
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    fmat = orc.phase_matrix(track[0], x, f)
    a = fmat[:, cols] if cols_dict is None else fmat @ cols_dict(cols)   # K x |cols|
    g_ref = a.conj().T @ a
    b_ref = a.conj().T @ d
    rr, cc = np.meshgrid(cols, cols, indexing="ij")
    got = g.gram_entries(rr.ravel(), cc.ravel()).reshape(cols.size, cols.size)
    assert_close(got, g_ref, 1e-4, "gram entries")
    b = g.b()
    assert_close(b[cols], b_ref, 1e-4, "b")
    st = g.state()
    assert abs(st["lambda"] - 0.05 * np.max(np.abs(b))) <= 1e-12 * st["lambda"]
    assert np.isfinite(st["lipschitz"]) and st["lipschitz"] > 0
    assert np.all(np.isfinite(g.coeffs()))
    xs = np.zeros(m, complex)
    xs[cols] = rng.standard_normal(cols.size) + 1j * rng.standard_normal(cols.size)
    y = g.gram_apply(xs)
    assert_close(y[cols], g_ref @ xs[cols], 1e-4, "gram apply")
    g.close()


def test_max_pixel_basis_scene():
    w = synth.Workload(name="max_512x256", nx=512, ny=256, n_freq=64,
                       f_lo_hz=9.9e9, f_hi_hz=10.1e9, n_pulses=8, span_deg=20.0,
                       seed=12)
    assert w.m_atoms == 131072
    _check(w, None)


def test_max_gaussian_atoms():
    w = synth.Workload(name="max_atoms_32x32", nx=32, ny=32, n_freq=64,
                       f_lo_hz=9.9e9, f_hi_hz=10.1e9, n_pulses=8, span_deg=20.0,
                       dictionary="gaussian", n_atoms=131072, dict_seed=5, seed=13)
    _check(w, lambda cols: synth.gaussian_dictionary_columns(w.n_pixels, cols, w.dict_seed))
