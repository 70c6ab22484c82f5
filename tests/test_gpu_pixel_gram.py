"""Pixel-space Gram form (pixel_gram): with A_s = F_s H, the context keeps
P_n = sum F_s^H F_s and b_pix = sum F_s^H d_s and applies G_n = H^H P_n H as
H^H (P_n (H x)).  Parity against the FP64 oracle run with the edgelet
dictionary itself (stored G_n, Eqs. 12-13 and Algorithm 1): every pulse,
the experiments' two dictionaries and a diagonal one, all three precisions;
H^H P_n H against the oracle's G_n, H^H b_pix against its b_n, lambda_n,
L_n, the coefficients and the stop rule's step counts.  Also: the stored-
Gram edgelet form to rounding, the simulated data, and the calls this form
does not offer.  (tests/test_oracle_pins.py pins G_n = H^H P_n H on the
oracle.)"""
import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, rel_err, oracle_config,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

TOL = {
    "fp64": {"gram": 1e-9, "b": 1e-9, "c": 1e-7},
    "fp32": {"gram": 2e-6, "b": 2e-6, "c": 1e-4},
    "split_bf16": {"gram": 1e-4, "b": 1e-4, "c": 1e-3},
}

DICTS = {
    "squares": ((4,), (0.0, 90.0)),
    "lines": ((2, 4, 6), (0.0,)),
    "diagonal": ((3,), (45.0, 135.0)),
}


def _w(name, nx=12, ny=12, n_freq=40, n_pulses=5, seed=9):
    lengths, angles = DICTS[name]
    return small_workload(nx=nx, ny=ny, n_freq=n_freq, n_pulses=n_pulses,
                          dictionary="edgelet", edgelet_lengths=lengths,
                          edgelet_angles=angles, sparsity=0.02, seed=seed)


def _ctx(w, prec, pixel=True):
    cfg = gpu_config(w, prec)
    cfg.pixel_gram = 1 if pixel else 0
    return osar.Osar(cfg)


def _run(w, prec, steps, tol=0.0, check=None):
    track, dic, _, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    g = _ctx(w, prec)
    for s in range(track.shape[0]):
        of.push_pulse(track[s], data[s])
        g.push_pulse(track[s], data[s])
        no = of.iterate(steps, tol)
        ng = g.iterate(steps, tol)
        if check is not None:
            check(s, of, g, no, ng, dic)
    return of, g


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
@pytest.mark.parametrize("name", sorted(DICTS))
def test_pixel_gram_parity_every_pulse(prec, name):
    # 12 x 12 pixels (N = 144: 2 blocks), M = 288 / 432 / 288 atoms, K = 40
    w = _w(name)
    t = TOL[prec]

    def check(s, of, g, no, ng, h):
        p = g.gram()
        assert p.shape == (w.nx * w.ny, w.nx * w.ny)
        assert_close(h.conj().T @ p @ h, of.s.gram, t["gram"], "H^H P H")
        assert_close(g.b(), of.s.b, t["b"], "b")
        assert_coeffs(g.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec])
        st = g.state()
        assert st["n"] == of.s.n
        assert abs(st["lambda"] - of.s.lam) <= t["b"] * of.s.lam  # from b_n
        assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10
        assert st["t"] == pytest.approx(of.s.t, rel=1e-12)

    _run(w, prec, steps=10, check=check)


def test_pixel_gram_stop_rule_counts():
    w = _w("lines", n_pulses=6, seed=4)

    def check(s, of, g, no, ng, h):
        assert ng == no
        assert_coeffs(g.coeffs(), of.s, TOL["fp64"]["c"], SUPPORT_DELTA["fp64"])

    _run(w, "fp64", steps=30, tol=1e-4, check=check)


def test_pixel_gram_against_the_stored_gram_form():
    # 32 x 32 pixels, the square dictionary: M = 2048 (16 blocks), N = 1024
    w = _w("squares", nx=32, ny=32, n_freq=64, n_pulses=4, seed=12)
    track, _, _, data = build_problem(w)
    a, b = _ctx(w, "split_bf16", pixel=False), _ctx(w, "split_bf16", pixel=True)
    assert a.m_atoms == b.m_atoms == 2048
    for s in range(track.shape[0]):
        for g in (a, b):
            g.push_pulse(track[s], data[s])
            g.iterate(12, 0.0, want_count=False)
        assert rel_err(b.coeffs(), a.coeffs()) <= 1e-4
        assert rel_err(b.b(), a.b()) <= 1e-5
        sa, sb = a.state(), b.state()
        assert abs(sa["lipschitz"] - sb["lipschitz"]) <= 1e-5 * sa["lipschitz"]
    assert b.device_bytes() < a.device_bytes()


def test_pixel_gram_simulated_pulse_matches_the_oracle():
    w = _w("lines", nx=10, ny=7, n_freq=24)
    track, dic, c_true, _ = build_problem(w)
    g = _ctx(w, "fp64")
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    for s in (0, 3):
        want = orc.simulate_pulse(orc.forward_block(orc.phase_matrix(track[s], x, f), dic),
                                  c_true)
        assert rel_err(g.simulate_pulse(track[s], c_true), want) <= 1e-9


def test_pixel_gram_refuses_what_it_does_not_offer(tmp_path):
    w = _w("squares", n_pulses=2)
    track, _, _, data = build_problem(w)
    g = _ctx(w, "split_bf16")
    g.push_pulse(track[0], data[0])
    g.iterate(3)
    with pytest.raises(osar.OsarError) as e:
        g.save(str(tmp_path / "ck.bin"))
    assert e.value.status == osar.OSAR_E_STATE
    with pytest.raises(osar.OsarError) as e:
        g.lambda_state(0)
    assert e.value.status == osar.OSAR_E_STATE
    # the context stays usable
    g.push_pulse(track[1], data[1])
    assert g.iterate(3) == 3


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_pixel_gram_non_white_pulses(prec):
    # Eq. 12 with R_n = diag(variances): P_n = sum F^H R^-1 F and b_pix =
    # sum F^H R^-1 d keep the factorisation, white and non-white pulses mixed
    w = _w("squares", n_pulses=6, seed=21)
    track, dic, _, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    g = _ctx(w, prec)
    rng = np.random.default_rng(3)
    t = TOL[prec]
    for s in range(track.shape[0]):
        var = None if s % 3 == 2 else rng.uniform(0.3, 3.0, w.n_freq)
        of.push_pulse(track[s], data[s], var)
        g.push_pulse(track[s], data[s], var)
        of.iterate(10)
        g.iterate(10, want_count=False)
        assert_close(dic.conj().T @ g.gram() @ dic, of.s.gram, t["gram"], "H^H P H")
        assert_close(g.b(), of.s.b, t["b"], "b")
        assert_coeffs(g.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec])
        st = g.state()
        assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10


# --------------------------------------------------------------------------
# Dense dictionaries (Gaussian, host): G_n = D^H P_n D applied as
# D^H (P_n (D x)), the two dictionary products as matrix-vector kernels.

def _wg(nx=12, ny=12, n_freq=40, n_pulses=5, m=300, seed=19, dict_seed=7):
    return small_workload(nx=nx, ny=ny, n_freq=n_freq, n_pulses=n_pulses,
                          dictionary="gaussian", n_atoms=m, sparsity=0.03,
                          seed=seed, dict_seed=dict_seed)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_dense_pixel_gram_parity_every_pulse(prec):
    # 12 x 12 pixels (N = 144: 2 blocks), M = 300 Gaussian atoms (ragged), K = 40
    w = _wg()
    t = TOL[prec]

    def check(s, of, g, no, ng, dic):
        p = g.gram()
        assert p.shape == (w.nx * w.ny, w.nx * w.ny)
        assert_close(dic.conj().T @ p @ dic, of.s.gram, t["gram"], "D^H P D")
        assert_close(g.b(), of.s.b, t["b"], "b")
        assert_coeffs(g.coeffs(), of.s, t["c"], SUPPORT_DELTA[prec])
        st = g.state()
        assert st["n"] == of.s.n
        assert abs(st["lambda"] - of.s.lam) <= t["b"] * of.s.lam
        assert abs(st["lipschitz"] - of.s.lip) <= max(t["gram"], 1e-7) * of.s.lip * 10
        assert st["t"] == pytest.approx(of.s.t, rel=1e-12)

    _run(w, prec, steps=10, check=check)


def test_dense_pixel_gram_host_dictionary_and_stop_rule():
    w = _wg(nx=10, ny=9, m=200, n_pulses=5, seed=23)
    track, dic, _, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    cfg = gpu_config(w, "fp64", host_dictionary=dic)
    cfg.pixel_gram = 1
    g = osar.Osar(cfg)
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
        g.push_pulse(track[s], data[s])
        assert g.iterate(40, 1e-5) == of.iterate(40, 1e-5)
        assert_coeffs(g.coeffs(), of.s, TOL["fp64"]["c"], SUPPORT_DELTA["fp64"])


def test_dense_pixel_gram_against_the_stored_gram_form():
    # 32 x 32 pixels, M = 2048 Gaussian atoms (16 blocks), N = 1024
    w = _wg(nx=32, ny=32, n_freq=64, n_pulses=4, m=2048, seed=12)
    track, _, _, data = build_problem(w)
    a, b = _ctx(w, "split_bf16", pixel=False), _ctx(w, "split_bf16", pixel=True)
    for s in range(track.shape[0]):
        for g in (a, b):
            g.push_pulse(track[s], data[s])
            g.iterate(12, 0.0, want_count=False)
        # the two forms round differently (split products of F D against
        # split F and split D products): within the split-BF16 bars
        assert rel_err(b.coeffs(), a.coeffs()) <= 1e-4
        assert rel_err(b.b(), a.b()) <= 1e-5
        sa, sb = a.state(), b.state()
        assert abs(sa["lipschitz"] - sb["lipschitz"]) <= 1e-4 * sa["lipschitz"]
    assert b.device_bytes() < a.device_bytes()


def test_dense_pixel_gram_simulated_pulse_matches_the_oracle():
    w = _wg(nx=10, ny=7, n_freq=24, m=150)
    track, dic, c_true, _ = build_problem(w)
    g = _ctx(w, "fp64")
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    for s in (0, 3):
        want = orc.simulate_pulse(orc.forward_block(orc.phase_matrix(track[s], x, f), dic),
                                  c_true)
        assert rel_err(g.simulate_pulse(track[s], c_true), want) <= 1e-9
