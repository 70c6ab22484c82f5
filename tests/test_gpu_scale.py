"""Parity at the sizes the bench runs: the split-BF16 path with the bench's
launch configuration (SM-pair tensor-core products, the first power step in
the Gram update's epilogue, the last power step fused with the first FISTA
step, overlapped synthesis, the Gram update run ahead into the second Gram
buffer on part of the GPU: gram_ahead = 2, so that it runs ahead on every
push even after the synchronising iterate) against the FP64 oracle after
every pulse's 20-step burst (Algorithm 1; Eqs. 11-13), on problems large
enough that every multi-tile path runs:

* 64 x 64 pixels, M = 8192 Gaussian atoms, K = 512: 2080 packed Gram blocks,
  so each SM pair of the Gram update handles many tiles (TMEM double buffer,
  the epilogue's prefetch across tile boundaries, the fused power step's
  tile-parity reduction buffers) and the matvec hands out segment tickets;
* the 128 x 128 / M = 32768 / K = 512 workload itself (its first pulses),
  in the stored-Gram form and in the pixel-space Gram form (P_n, N x N,
  G_n applied as D^H P_n D);
* the 256 x 256 pixel-basis workload (M = 65536, K = 1024, 10 steps per
  pulse; its first pulses), against the oracle in its matrix-free mode
  (Eq. 10: A_n x = sum_k G_k^H G_k x), since the 69 GB FP64 Gram does not
  fit in host memory.

Bars (split-BF16, as in test_gpu_parity): b and sampled Gram entries <= 1e-4,
coefficients <= 1e-3, each as a relative 2-norm and as a worst element
relative to the largest reference entry; no support difference outside the
threshold band (SUPPORT_DELTA); L_n within 1e-3, lambda_n within 1e-3 and t
within 1e-9 (relative)."""
import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar, synth
from tests.helpers import (oracle_config, assert_close, assert_coeffs,
                           SUPPORT_DELTA, host_gaussian_dictionary,
                           dictionary_pulses)
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

TOL_GRAM, TOL_B, TOL_C = 1e-4, 1e-4, 1e-3


def _mid_workload():
    return synth.Workload(
        name="mid_64x64_M8192", nx=64, ny=64, n_freq=512, f_lo_hz=9.75e9,
        f_hi_hz=10.25e9, n_pulses=64, span_deg=45.0, dictionary="gaussian",
        n_atoms=8192, dict_seed=2, sparsity=0.03, snr_db=25.0, seed=9)


def _sampled_entries(m, rng, k=48):
    # random atoms plus both sides of block and matrix edges
    cols = np.unique(np.concatenate([
        rng.choice(m, k, replace=False),
        [0, 1, 127, 128, 255, 256, m // 2 - 1, m // 2, m - 129, m - 128, m - 1]]))
    rr, cc = np.meshgrid(cols, cols, indexing="ij")
    return rr.ravel(), cc.ravel()


def _compare(of, gpu, rng, what):
    assert_close(gpu.b(), of.s.b, TOL_B, f"{what} b")
    rows, cols = _sampled_entries(of.m, rng)
    ref = (of.s.gram.entries(rows, cols) if of.matrix_free
           else of.s.gram[rows, cols])
    assert_close(gpu.gram_entries(rows, cols), ref, TOL_GRAM, f"{what} gram entries")
    st = gpu.state()
    assert st["n"] == of.s.n
    assert abs(st["lambda"] - of.s.lam) <= 1e-3 * of.s.lam, (what, st, of.s.lam)
    assert abs(st["lipschitz"] - of.s.lip) <= 1e-3 * of.s.lip, (what, st, of.s.lip)
    assert abs(st["t"] - of.s.t) <= 1e-9 * of.s.t, (what, st, of.s.t)
    return assert_coeffs(gpu.coeffs(), of.s, TOL_C, SUPPORT_DELTA["split_bf16"],
                         f"{what} c")


def _run(w, pulses, steps, rng, pixel_form=False):
    """The stored-Gram context (and, with pixel_form, the pixel-space Gram
    form of the same dictionary beside it) against one oracle run."""
    dic = host_gaussian_dictionary(w.n_pixels, w.m_atoms, w.dict_seed)
    track, _, data = dictionary_pulses(w, dic, pulses)
    of = orc.OnlineFista(oracle_config(w, dic, lam=w.lambda_rel))
    cfg = gpu_config(w, "split_bf16", lam=w.lambda_rel)
    cfg.gram_ahead = 2
    gpu = osar.Osar(cfg)
    pix = None
    if pixel_form:
        cfg = gpu_config(w, "split_bf16", lam=w.lambda_rel)
        cfg.pixel_gram = 1
        pix = osar.Osar(cfg)
    errs = []
    for s in range(pulses):
        of.push_pulse(track[s], data[s])
        for g in (gpu, pix):
            if g is not None:
                g.push_pulse(track[s], data[s])
                assert g.iterate(steps) == steps
        assert of.iterate(steps) == steps
        errs.append(_compare(of, gpu, rng, f"pulse {s}"))
        if pix is not None:
            assert_close(pix.b(), of.s.b, TOL_B, f"pulse {s} pixel form b")
            st = pix.state()
            assert abs(st["lipschitz"] - of.s.lip) <= 1e-3 * of.s.lip
            assert abs(st["lambda"] - of.s.lam) <= 1e-3 * of.s.lam
            errs.append(assert_coeffs(pix.coeffs(), of.s, TOL_C,
                                      SUPPORT_DELTA["split_bf16"],
                                      f"pulse {s} pixel form c"))
    assert gpu.profile_ahead() == pulses
    # the matvec on a dense random vector, every row
    x = rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms)
    assert_close(gpu.gram_apply(x), of.s.gram @ x, TOL_GRAM, "gram apply")
    if pix is not None:
        assert pix.device_bytes() < 0.6 * gpu.device_bytes()
        pix.close()
    return of, gpu, errs


def test_multi_tile_64x64_M8192_every_pulse():
    w = _mid_workload()
    of, gpu, errs = _run(w, pulses=5, steps=20, rng=np.random.default_rng(1))
    # the whole Gram at the end
    assert_close(gpu.gram(), of.s.gram, TOL_GRAM, "gram")
    print("64x64 M=8192 split-BF16 coefficient errors per pulse:",
          " ".join(f"{e:.2e}" for e in errs))


def test_headline_128x128_M32768_first_pulses():
    w = synth.workloads()["c2_128x128_split_bf16"]
    of, gpu, errs = _run(w, pulses=3, steps=20, rng=np.random.default_rng(2),
                         pixel_form=True)
    print("128x128 M=32768 split-BF16 coefficient errors per pulse "
          "(stored form, pixel-space form):", " ".join(f"{e:.2e}" for e in errs))


def test_large_online_256x256_first_pulses_matrix_free_oracle():
    w = synth.workloads()["c5_256x256_split_bf16"]
    P, steps = 2, w.inner_steps
    track = synth.workload_track(w)[:P]
    c_true = synth.workload_scene(w)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    clean = np.stack([orc.phase_matrix(g, x, f) @ c_true for g in track])
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)[:P]
    data = clean + synth.scale_noise(clean, noise, w.snr_db)
    of = orc.OnlineFista(oracle_config(w, None, lam=w.lambda_rel), matrix_free=True)
    cfg = gpu_config(w, "split_bf16", lam=w.lambda_rel)
    cfg.gram_ahead = 2
    gpu = osar.Osar(cfg)
    rng = np.random.default_rng(3)
    errs = []
    for s in range(P):
        of.push_pulse(track[s], data[s])
        gpu.push_pulse(track[s], data[s])
        assert of.iterate(steps) == steps
        assert gpu.iterate(steps) == steps
        errs.append(_compare(of, gpu, rng, f"pulse {s}"))
    assert gpu.profile_ahead() == P
    xv = rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms)
    assert_close(gpu.gram_apply(xv), of.s.gram @ xv, TOL_GRAM, "gram apply")
    gpu.close()
    print("256x256 M=65536 split-BF16 coefficient errors per pulse:",
          " ".join(f"{e:.2e}" for e in errs))
