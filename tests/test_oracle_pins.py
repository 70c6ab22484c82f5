"""Pins for the FP64 oracle: each test checks it against something other than
itself (closed forms, invariants, an independent solver, brute force, values
evaluated by hand from the paper's Table I)."""
import json
import os

import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import synth
from tests.helpers import small_workload, build_problem, oracle_config, rel_err

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- phases ---

def test_phase_entries_unit_modulus_and_exact_phase():
    """F[m,n] = exp(-i 2 k_m R_n) (Eqs. 2-4): |F| = 1 and the phase equals the
    40-digit value of -4 pi f_m R_n / c mod 2 pi, where R_n is evaluated in
    40-digit arithmetic from the same FP64 coordinates."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    w = synth.workloads()["c2_128x128_split_bf16"]
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    gamma = synth.workload_track(w)[77]
    rng = np.random.default_rng(5)
    ms = rng.integers(0, w.n_freq, 40)
    ns = rng.integers(0, w.n_pixels, 40)
    fm = orc.phase_matrix(gamma, x[ns], f[ms])
    two_pi = 2 * mp.pi
    worst = 0.0
    for q in range(40):
        val = fm[q, q]
        assert abs(abs(val) - 1.0) < 1e-14
        r = mp.sqrt(sum((mp.mpf(float(gamma[a])) - mp.mpf(float(x[ns[q], a]))) ** 2
                        for a in range(3)))
        theta = -4 * mp.pi * mp.mpf(float(f[ms[q]])) * r / mp.mpf(orc.C_LIGHT)
        exact = float(mp.fmod(theta, two_pi))
        got = float(np.angle(val))
        diff = (got - exact + np.pi) % (2 * np.pi) - np.pi
        worst = max(worst, abs(diff))
    # FP64 rounding of a ~5e5 rad argument is ~1e-10 rad
    assert worst < 2e-9, worst


def test_pixel_grid_and_frequencies():
    x = orc.pixel_positions(4, 3, 2.0)
    assert x.shape == (12, 3)
    np.testing.assert_array_equal(x[0], [-3.0, -2.0, 0.0])
    np.testing.assert_array_equal(x[5], [-1.0, 0.0, 0.0])    # i=1, j=1
    np.testing.assert_array_equal(x[11], [3.0, 2.0, 0.0])
    f = orc.frequencies(5, 1.0, 2.0)
    np.testing.assert_allclose(f, [1.0, 1.25, 1.5, 1.75, 2.0])


# ------------------------------------------------------- Gram recursion ---

@pytest.mark.parametrize("dictionary", ["identity", "gaussian"])
def test_recursion_equals_batch_gram_and_data(dictionary):
    """Eq. 13's recursion equals the stacked (batch) Gram and data vector, and
    G c - b equals the matrix-free gradient of Eq. 10."""
    w = small_workload(nx=6, ny=5, n_freq=12, n_pulses=9,
                       dictionary=dictionary,
                       n_atoms=45 if dictionary == "gaussian" else None)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    blocks = []
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
        blocks.append(of.block(track[s]))
    gb = orc.batch_gram(blocks)
    bb = orc.batch_data(blocks, list(data))
    assert rel_err(of.s.gram, gb) < 1e-12
    assert rel_err(of.s.b, bb) < 1e-12
    y = synth.sparse_coefficients(of.m, 0.3, np.random.default_rng(3))
    assert rel_err(of.s.gram @ y - of.s.b,
                   orc.gradient_matrix_free(blocks, list(data), y)) < 1e-12


def test_identity_gram_closed_form():
    """Pixel basis: G_jj = n K exactly and the off-diagonal entries are the
    Dirichlet-kernel sum over pulses of
    exp(i(2k0 + (K-1)dk) dR) sin(K dk dR) / sin(dk dR), dR = R_i - R_j."""
    w = small_workload(nx=7, ny=6, n_freq=24, n_pulses=11, span_deg=20.0)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None))
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
    g = of.s.gram
    nk = w.n_pulses * w.n_freq
    np.testing.assert_allclose(np.real(np.diag(g)), nk, rtol=1e-13, atol=0)
    np.testing.assert_allclose(np.imag(np.diag(g)), 0.0, atol=1e-10)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    k0 = 2 * np.pi * w.f_lo_hz / orc.C_LIGHT
    dk = 2 * np.pi * (w.f_hi_hz - w.f_lo_hz) / ((w.n_freq - 1) * orc.C_LIGHT)
    kk = w.n_freq
    closed = np.zeros_like(g)
    for gamma in track:
        r = orc.ranges(gamma, x)
        dr = r[:, None] - r[None, :]
        s = np.sin(dk * dr)
        with np.errstate(invalid="ignore", divide="ignore"):
            ratio = np.where(np.abs(s) < 1e-300, kk, np.sin(kk * dk * dr) / s)
        closed += np.exp(1j * (2 * k0 + (kk - 1) * dk) * dr) * ratio
    assert np.max(np.abs(g - closed)) / nk < 1e-8


def test_gram_hermitian_psd():
    w = small_workload(nx=5, ny=5, n_freq=8, n_pulses=4,
                       dictionary="gaussian", n_atoms=50)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
    g = of.s.gram
    assert np.linalg.norm(g - g.conj().T) <= 1e-14 * np.linalg.norm(g)
    ev = np.linalg.eigvalsh(0.5 * (g + g.conj().T))
    # rank <= K P = 32 < M = 50: PSD with a null space
    assert ev.min() >= -1e-12 * ev.max()
    assert np.sum(ev > 1e-9 * ev.max()) <= w.n_freq * w.n_pulses


# ------------------------------------------------------------ Lipschitz ---

def test_power_iteration_bounds_and_convergence():
    """mu <= lambda_max (Eq. 11), converges to it, and stays under the
    incremental bound of Eq. 14."""
    w = small_workload(nx=6, ny=6, n_freq=16, n_pulses=8)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None, power_iters_first=40,
                                       power_iters=40, margin=0.0))
    bound = 0.0
    for s in range(w.n_pulses):
        a_s = of.block(track[s])
        bound = orc.incremental_lipschitz_bound(bound, a_s)
        of.push_pulse(track[s], data[s])
        lmax = np.linalg.eigvalsh(of.s.gram).max()
        assert of.s.lip <= lmax * (1 + 1e-12)
        assert lmax <= bound * (1 + 1e-12)
    mu, _ = orc.power_iteration(of.s.gram, of.s.v, 2000)
    assert abs(mu - np.linalg.eigvalsh(of.s.gram).max()) <= 1e-10 * mu


# ------------------------------------------------------------- shrinkage ---

def test_soft_threshold_table():
    u = np.array([3 + 4j, 3 + 4j, 3 + 4j, 0j, -2j, 1e-300 + 0j])
    a = [1.0, 5.0, 5.0 - 1e-9, 0.5, 2.0, 0.0]
    out = np.array([orc.soft_threshold(np.array([ui]), ai)[0]
                    for ui, ai in zip(u, a)])
    np.testing.assert_allclose(out[0], 2.4 + 3.2j, rtol=0, atol=1e-15)
    assert out[1] == 0                      # |u| == alpha: exactly zero
    np.testing.assert_allclose(abs(out[2]), 1e-9, rtol=1e-6)
    assert out[3] == 0                      # u = 0
    assert out[4] == 0                      # |u| == alpha
    assert out[5] == u[5]                   # alpha = 0: identity


def test_soft_threshold_is_the_prox_by_brute_force():
    """S_a(u) minimises 1/2 |x - u|^2 + a |x| over a fine grid of x in C."""
    rng = np.random.default_rng(7)
    grid = np.linspace(-3, 3, 1201)
    xr, xi = np.meshgrid(grid, grid, indexing="ij")
    xc = xr + 1j * xi
    for _ in range(6):
        u = complex(rng.uniform(-2, 2), rng.uniform(-2, 2))
        a = float(rng.uniform(0.1, 1.5))
        obj = 0.5 * np.abs(xc - u) ** 2 + a * np.abs(xc)
        best = xc.flat[np.argmin(obj)]
        s = orc.soft_threshold(np.array([u]), a)[0]
        assert abs(best - s) <= 2 * (grid[1] - grid[0])
        # phase is kept, modulus shrinks by a
        if s != 0:
            assert abs(abs(s) - (abs(u) - a)) < 1e-14
            assert abs(np.angle(s) - np.angle(u)) < 1e-12


# ---------------------------------------------------------------- FISTA ---

def _tiny_problem(seed=0):
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=16, seed=seed)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None))
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
    return w, of, c_true


def _coordinate_descent(g, b, lam, sweeps):
    """Independent LASSO solver: cyclic complex coordinate descent,
    c_i <- S_lambda(b_i - sum_{j != i} G_ij c_j) / G_ii."""
    c = np.zeros_like(b)
    gc = np.zeros_like(b)
    for _ in range(sweeps):
        for i in range(b.size):
            r = b[i] - (gc[i] - g[i, i] * c[i])
            new = orc.soft_threshold(np.array([r]), lam)[0] / g[i, i].real
            delta = new - c[i]
            if delta != 0:
                gc += g[:, i] * delta
                c[i] = new
    return c


def test_fista_reaches_kkt_solution_and_matches_coordinate_descent():
    w, of, c_true = _tiny_problem()
    g, b, lam = of.s.gram, of.s.b, of.s.lam
    lmax = np.linalg.eigvalsh(g).max()
    lmin = np.linalg.eigvalsh(g).min()
    assert lmin > 0                              # unique minimiser
    c, _, _ = orc.fista_fixed(g, b, lam, lmax, 20000)
    assert orc.kkt_residual(g, b, c, lam) < 1e-9
    c_cd = _coordinate_descent(g, b, lam, 400)
    assert orc.kkt_residual(g, b, c_cd, lam) < 1e-9
    assert rel_err(c, c_cd) < 1e-8


def test_fista_minimum_by_random_perturbation():
    """Brute force: no perturbation of the FISTA point lowers Eq. 8."""
    w, of, c_true = _tiny_problem(seed=4)
    g, b, lam = of.s.gram, of.s.b, of.s.lam
    c, _, _ = orc.fista_fixed(g, b, lam, np.linalg.eigvalsh(g).max(), 20000)
    j0 = orc.lasso_objective_gram(g, b, c, lam)
    rng = np.random.default_rng(1)
    for scale in (1e-1, 1e-3, 1e-5):
        d = scale * (rng.standard_normal((400, c.size))
                     + 1j * rng.standard_normal((400, c.size)))
        for k in range(d.shape[0]):
            assert orc.lasso_objective_gram(g, b, c + d[k], lam) >= j0 - 1e-9 * abs(j0)


def test_gram_objective_equals_data_objective():
    """Eq. 8 through (G, b) equals Eq. 8 through the stored pulses."""
    w = small_workload(nx=5, ny=4, n_freq=10, n_pulses=5)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None))
    blocks = []
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
        blocks.append(of.block(track[s]))
    c = c_true * 0.7 + 0.01
    const = 0.5 * float(np.sum(np.abs(data) ** 2))
    j_gram = orc.lasso_objective_gram(of.s.gram, of.s.b, c, 0.3, const)
    j_data = orc.lasso_objective(blocks, list(data), c, 0.3)
    assert abs(j_gram - j_data) <= 1e-10 * abs(j_data)


def test_fista_beck_teboulle_rate():
    """With t_1 = 1: F(c_k) - F* <= 2 L |c_0 - c*|^2 / (k+1)^2."""
    w, of, c_true = _tiny_problem(seed=2)
    g, b, lam = of.s.gram, of.s.b, of.s.lam
    lip = np.linalg.eigvalsh(g).max()
    c_star = _coordinate_descent(g, b, lam, 600)
    f_star = orc.lasso_objective_gram(g, b, c_star, lam)
    _, _, hist = orc.fista_fixed(g, b, lam, lip, 300)
    r0 = np.linalg.norm(c_star) ** 2
    for k, ck in enumerate(hist, start=1):
        gap = orc.lasso_objective_gram(g, b, ck, lam) - f_star
        assert gap <= 2 * lip * r0 / (k + 1) ** 2 + 1e-9 * abs(f_star)


def test_momentum_sequence():
    t = 1.0
    for k in range(1, 200):
        assert t >= (k + 1) / 2.0 - 1e-12
        tn = orc.momentum_next(t)
        assert abs(tn * tn - tn - t * t) < 1e-9 * tn * tn   # t'^2 - t' = t^2
        t = tn


# ---------------------------------------------------------- point target ---

def test_point_target_closed_form():
    """Noise-free single scatterer in the pixel basis: the LASSO minimiser is
    c* = a (1 - lambda / (|a| G_jj)) e_j."""
    w = small_workload(nx=7, ny=7, n_freq=16, n_pulses=12, snr_db=300.0)
    j = 17
    a = 0.8 * np.exp(0.7j)
    c_true = np.zeros(w.n_pixels, dtype=np.complex128)
    c_true[j] = a
    track, dic, _, data = build_problem(w, noise=False, c_true=c_true)
    lam = 10.0
    of = orc.OnlineFista(oracle_config(w, None, lam=lam, lambda_relative=False))
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
    g, b = of.s.gram, of.s.b
    gjj = g[j, j].real
    expect = np.zeros_like(c_true)
    expect[j] = a * (1.0 - lam / (abs(a) * gjj))
    assert orc.kkt_residual(g, b, expect, lam) < 1e-10
    c, _, _ = orc.fista_fixed(g, b, lam, np.linalg.eigvalsh(g).max(), 5000)
    assert np.max(np.abs(c - expect)) < 1e-9


def test_online_point_targets_land_on_their_pixels():
    w = small_workload(nx=16, ny=16, n_freq=32, n_pulses=24, span_deg=40.0,
                       snr_db=30.0, seed=9)
    c_true = np.zeros(w.n_pixels, dtype=np.complex128)
    pix = [3 * 16 + 3, 8 * 16 + 12, 13 * 16 + 5]
    c_true[pix] = [0.9, 0.8j, -0.7]
    track, dic, _, data = build_problem(w, c_true=c_true)
    of, _ = orc.run_online(oracle_config(w, None, lam=0.1), track, data, 20)
    top = set(np.argsort(-np.abs(of.s.c_hat))[:3].tolist())
    assert top == set(pix)


# ---------------------------------------------------------- online burst ---

def test_iterate_split_equals_single_burst():
    w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=5)
    track, dic, c_true, data = build_problem(w)
    a = orc.OnlineFista(oracle_config(w, None))
    b = orc.OnlineFista(oracle_config(w, None))
    for s in range(w.n_pulses):
        a.push_pulse(track[s], data[s])
        b.push_pulse(track[s], data[s])
        a.iterate(7)
        b.iterate(3)
        b.iterate(4)
        assert np.array_equal(a.s.c_hat, b.s.c_hat)
        assert a.s.t == b.s.t


def test_momentum_carried_vs_restart():
    w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=4)
    track, dic, c_true, data = build_problem(w)
    carry, _ = orc.run_online(oracle_config(w, None), track, data, 5)
    rest, _ = orc.run_online(oracle_config(w, None, restart_momentum=True),
                             track, data, 5)
    t = 1.0
    for _ in range(20):
        t = orc.momentum_next(t)
    assert abs(carry.s.t - t) < 1e-12              # 4 bursts x 5 steps, carried
    t = 1.0
    for _ in range(5):
        t = orc.momentum_next(t)
    assert abs(rest.s.t - t) < 1e-12


def _hand_fista_2x2(g, b, lam, lip, t1, steps):
    """Algorithm 1's inner loop on a 2 x 2 problem in scalar complex
    arithmetic (no oracle function): returns per step the iterate c_k, the
    point z_k where the gradient was taken, the momentum point z_{k+1} and the
    previous iterate c_{k-1}."""
    tau = 1.0 / lip
    c_prev = [0j, 0j]
    z = [0j, 0j]
    t = t1
    out = []
    for _ in range(steps):
        grad = [g[0][0] * z[0] + g[0][1] * z[1] - b[0],
                g[1][0] * z[0] + g[1][1] * z[1] - b[1]]
        u = [z[i] - tau * grad[i] for i in range(2)]
        c = []
        for ui in u:
            a = abs(ui)
            c.append(ui * (1.0 - lam * tau / a) if a > lam * tau else 0j)
        t_next = (1.0 + (1.0 + 4.0 * t * t) ** 0.5) / 2.0
        beta = (t - 1.0) / t_next
        z_next = [c[i] + beta * (c[i] - c_prev[i]) for i in range(2)]
        out.append({"c": c, "z": z, "z_next": z_next, "c_prev": c_prev})
        c_prev, z, t = c, z_next, t_next
    return out


def _norm2(v):
    return sum(abs(x) ** 2 for x in v) ** 0.5


def test_tolerance_stop_rule_by_hand():
    """The burst stops at the first step k with |c^(k) - z^(k)| <= tol |c^(k)|,
    z^(k) the point where step k took its gradient.  The gaps are computed by
    hand on a 2 x 2 Hermitian problem; tol is placed so that the two plausible
    misreadings (|c^(k) - c^(k-1)|, or the post-momentum point z^(k+1)) stop
    at other steps, so either would fail here."""
    g = [[2.0 + 0j, 0.5 - 0.5j], [0.5 + 0.5j, 1.0 + 0j]]
    b = [1.0 + 1.0j, -0.5 + 0.2j]
    lam, lip = 0.1, 3.0
    steps = _hand_fista_2x2(g, b, lam, lip, 1.0, 40)

    def first_stop(gap, tol):
        for k, st in enumerate(steps):
            if gap(st) <= tol * _norm2(st["c"]):
                return k + 1
        return None

    right = lambda st: _norm2([st["c"][i] - st["z"][i] for i in range(2)])
    prev = lambda st: _norm2([st["c"][i] - st["c_prev"][i] for i in range(2)])
    post = lambda st: _norm2([st["c"][i] - st["z_next"][i] for i in range(2)])
    tol = None
    for cand in np.geomspace(1e-1, 1e-8, 200):
        k = first_stop(right, cand)
        if k is not None and k > 2 and first_stop(prev, cand) != k \
                and first_stop(post, cand) != k:
            tol = float(cand)
            break
    assert tol is not None, "no tolerance separates the three readings"
    k_star = first_stop(right, tol)

    of = orc.OnlineFista(orc.OracleConfig(nx=1, ny=2, pixel_m=1.0, n_freq=1,
                                          f_lo_hz=1e10, f_hi_hz=1e10,
                                          lam=lam, lambda_relative=False))
    of.s.gram = np.array(g, dtype=np.complex128)
    of.s.b = np.array(b, dtype=np.complex128)
    of.s.n, of.s.lip, of.s.lam = 1, lip, lam
    n = of.iterate(40, tol=tol)
    assert n == k_star
    assert np.allclose(of.s.c_hat, steps[k_star - 1]["c"], rtol=0, atol=1e-15)
    assert of.iterate(10, tol=tol) == 0            # a converged burst stays put
    # the gap at the stop is below tol, the one before it above
    assert right(steps[k_star - 1]) <= tol * _norm2(steps[k_star - 1]["c"])
    assert right(steps[k_star - 2]) > tol * _norm2(steps[k_star - 2]["c"])


def test_tolerance_stop_point_is_near_optimal():
    """At the stop, c = prox(z - tau grad f(z)) gives (G - L I)(c - z) as an
    element of grad f(c) + lambda d|c|_1, so the oracle's KKT residual (max
    violation / lambda) is at most L |c - z| / lambda <= L tol |c| / lambda
    when 0 <= G <= L I."""
    w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=6)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None))
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
    # the step size of the bound: L >= lambda_max(G)
    of.s.lip = 1.01 * float(np.linalg.eigvalsh(of.s.gram).max())
    tol = 1e-10
    n = of.iterate(200000, tol=tol)
    assert 0 < n < 200000
    c = of.s.c_hat
    bound = of.s.lip * tol * np.linalg.norm(c) / of.s.lam
    kkt = orc.kkt_residual(of.s.gram, of.s.b, c, of.s.lam)
    assert kkt <= bound * (1 + 1e-6) + 1e-12, (kkt, bound)
    assert bound < 1e-6


# ------------------------------------------------- matrix-free Gram form ---

def test_matrix_free_online_fista_equals_the_stored_gram():
    """The matrix-free mode applies A_n x as sum_k G_k^H R_k^-1 (G_k x) (Eq. 10
    with Eqs. 12-13): its whole trajectory (L_n, lambda_n, t, c) equals the
    stored-Gram run up to summation order, white and non-white pulses mixed,
    and its entries equal the stored Gram's."""
    w = small_workload(nx=8, ny=6, n_freq=20, n_pulses=6, dictionary="gaussian",
                       n_atoms=70, seed=13, dict_seed=4)
    track, dic, c_true, data = build_problem(w)
    dense = orc.OnlineFista(oracle_config(w, dic))
    free = orc.OnlineFista(oracle_config(w, dic), matrix_free=True)
    rng = np.random.default_rng(2)
    for s in range(w.n_pulses):
        var = rng.uniform(0.5, 2.0, w.n_freq) if s % 2 else None
        for of in (dense, free):
            of.push_pulse(track[s], data[s], var)
            of.iterate(15)
        assert free.s.lip == pytest.approx(dense.s.lip, rel=1e-12)
        assert free.s.lam == pytest.approx(dense.s.lam, rel=1e-13)
        assert free.s.t == dense.s.t
        assert np.linalg.norm(free.s.c_hat - dense.s.c_hat) <= \
            1e-11 * np.linalg.norm(dense.s.c_hat)
    rows = np.array([0, 5, 69, 33, 12])
    cols = np.array([69, 5, 0, 7, 40])
    assert np.allclose(free.s.gram.entries(rows, cols), dense.s.gram[rows, cols],
                       rtol=0, atol=1e-12 * np.abs(dense.s.gram).max())
    x = rng.standard_normal(70) + 1j * rng.standard_normal(70)
    assert np.allclose(free.s.gram @ x, dense.s.gram @ x, rtol=0,
                       atol=1e-12 * np.abs(dense.s.gram @ x).max())


# ------------------------------------------------------- quality (§IV-B) ---

def test_large_coefficient_count_by_hand():
    c = np.array([0.03, -0.02, 0.02 + 0.001j, 0.5j, 0.0, -0.0199 - 0.0001j])
    # |c| = 0.03, 0.02, 0.020025, 0.5, 0, 0.01990025: strictly above 0.02
    assert orc.large_coefficient_count(c) == 3
    assert orc.large_coefficient_count(c, 0.0) == 5
    assert orc.large_coefficient_count(np.zeros(7)) == 0


def test_coefficient_snr_by_hand():
    # support {0, 1}: RMS sqrt((9 + 16) / 2); rest: sqrt((9e-4 + 16e-4) / 2);
    # ratio 100 -> exactly 40 dB
    c = np.array([3.0, 4.0j, 0.03, -0.04j])
    assert orc.coefficient_snr_db(c, [0, 1]) == pytest.approx(40.0, abs=1e-12)
    # duplicates in the support change nothing; an empty complement is +inf
    assert orc.coefficient_snr_db(c, [1, 0, 1]) == pytest.approx(40.0, abs=1e-12)
    assert orc.coefficient_snr_db(c, [0, 1, 2, 3]) == float("inf")
    # equal RMS on both sides: 0 dB
    assert orc.coefficient_snr_db(np.array([1.0, 1j, -1.0, 0.6 + 0.8j]),
                                  [0, 3]) == pytest.approx(0.0, abs=1e-12)


# ------------------------------------------------------------- Table I ---

def test_memory_table_golden():
    g = json.load(open(os.path.join(HERE, "golden", "table1_memory.json")))
    for case in g["cases"]:
        fista, online = orc.memory_values(case["M"], case["N"], case["N_r"],
                                          case["n"])
        assert fista == case["fista"]
        assert online == case["online"]


# ------------------------------------------------------- input generator ---

def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Random123)."""
    z = synth.philox4x32_10(np.zeros((1, 4), np.uint32), (0, 0))[0]
    assert [int(v) for v in z] == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    o = synth.philox4x32_10(np.full((1, 4), 0xFFFFFFFF, np.uint32),
                            (0xFFFFFFFF, 0xFFFFFFFF))[0]
    assert [int(v) for v in o] == [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    p = synth.philox4x32_10(
        np.array([[0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]], np.uint32),
        (0xa4093822, 0x299f31d0))[0]
    assert [int(v) for v in p] == [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_gaussian_dictionary_statistics():
    d = synth.gaussian_dictionary(256, 300, seed=3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), 1.0, rtol=1e-14)
    raw = d * np.sqrt(256)
    assert abs(np.mean(raw.real)) < 0.02 and abs(np.mean(raw.imag)) < 0.02
    assert abs(np.var(raw.real) - 0.5) < 0.02
    cols = synth.gaussian_dictionary_columns(256, np.array([7, 299]), seed=3)
    assert np.array_equal(cols, d[:, [7, 299]])


# ------------------------------------------------------------ edgelets ---
# §III-A: binary edgelets of length l and rotation psi centred at every pixel.
# The pins restate the atoms in closed form (a clipped run of columns or rows,
# or a hand-listed diagonal), not by the oracle's stepping rule.

def test_edgelet_atoms_horizontal_and_vertical_are_clipped_runs():
    nx, ny = 7, 5
    for l in (1, 2, 3, 4, 6):
        h = orc.edgelet_atoms(nx, ny, [l], [0.0])
        v = orc.edgelet_atoms(nx, ny, [l], [90.0])
        assert len(h) == len(v) == nx * ny
        back = (l - 1) // 2                      # pixels behind the centre
        for y in range(ny):
            for x in range(nx):
                lo, hi = max(0, x - back), min(nx - 1, x - back + l - 1)
                assert sorted(h[y * nx + x]) == [y * nx + c for c in range(lo, hi + 1)]
                lo, hi = max(0, y - back), min(ny - 1, y - back + l - 1)
                assert sorted(v[y * nx + x]) == [r * nx + x for r in range(lo, hi + 1)]


def test_edgelet_atoms_diagonals_by_hand():
    # 4 x 4 grid, length 3: offsets -1, 0, 1 along (1, 1) and (-1, 1)
    d45 = orc.edgelet_atoms(4, 4, [3], [45.0])
    assert sorted(d45[1 * 4 + 1]) == [0, 5, 10]          # (0,0) (1,1) (2,2)
    assert sorted(d45[0]) == [0, 5]                      # (-1,-1) dropped
    d135 = orc.edgelet_atoms(4, 4, [3], [135.0])
    assert sorted(d135[1 * 4 + 2]) == [3, 6, 9]          # (3,0) (2,1) (1,2)
    # length 4 along (1, 1) from (1, 1): offsets -1 .. 2
    assert sorted(orc.edgelet_atoms(4, 4, [4], [45.0])[5]) == [0, 5, 10, 15]


def test_edgelet_dictionary_counts_order_and_paper_square():
    nx = ny = 12
    lengths, angles = [2, 4, 6], [0.0]
    h = orc.edgelet_dictionary(nx, ny, lengths, angles)
    assert h.shape == (nx * ny, 3 * nx * ny)
    assert set(np.unique(h)) <= {0.0, 1.0}
    # atom m = (length index * rotations + rotation index) * N + y * nx + x
    m = (2 * 1 + 0) * nx * ny + 3 * nx + 5                 # length 6 at (5, 3)
    assert np.flatnonzero(h[:, m]).tolist() == [3 * nx + c for c in range(3, 9)]
    # dictionary 1 of the experiments (length 4, 0 and 90 degrees): a square
    # outline of side 4 with top-left (x0, y0) is exactly four atoms
    d1 = orc.edgelet_dictionary(nx, ny, [4], [0.0, 90.0])
    x0, y0, n = 3, 2, nx * ny
    c = np.zeros(2 * n)
    c[y0 * nx + x0 + 1] = 1                 # top edge, centre (x0 + 1, y0)
    c[(y0 + 3) * nx + x0 + 1] = 1           # bottom edge
    c[n + (y0 + 1) * nx + x0] = 1           # left edge, centre (x0, y0 + 1)
    c[n + (y0 + 1) * nx + x0 + 3] = 1       # right edge
    img = (d1 @ c).reshape(ny, nx)
    want = np.zeros((ny, nx))
    want[y0, x0:x0 + 4] += 1
    want[y0 + 3, x0:x0 + 4] += 1
    want[y0:y0 + 4, x0] += 1
    want[y0:y0 + 4, x0 + 3] += 1
    assert np.array_equal(img, want)


def test_paper_scenes_have_the_ideal_atom_counts():
    # §IV-A: the ideal numbers of coefficients are 4, 8, 5 and 5
    for kind, ideal, pixels in (("square", 4, 12), ("two_squares", 8, 24),
                                ("lines_spaced", 5, 22), ("lines_adjoined", 5, 22)):
        lengths, angles, c = synth.paper_scene(kind, 32, 32)
        assert np.count_nonzero(c) == ideal
        img = orc.edgelet_dictionary(32, 32, lengths, angles) @ c.real
        assert np.count_nonzero(img) == pixels
    # the pulse selection keeps about p of the positions, within the arc
    t = synth.sampled_track(1000, 4000.0, 1000.0, 2.0, 0.3, 7)
    assert 250 <= len(t) <= 350
    assert np.allclose(np.hypot(t[:, 0], t[:, 1]), 4000.0) and np.allclose(t[:, 2], 1000.0)


def test_pixel_space_gram_factors_the_dictionary_gram():
    # Eqs. 6 and 12-13 with A_s = F_s H: the pixel-basis statistics P_n =
    # sum F_s^H F_s and b_pix = sum F_s^H d_s give the dictionary's Gram and
    # data vector as H^H P_n H and H^H b_pix (the pixel-space Gram form)
    nx, ny = 6, 5
    h = orc.edgelet_dictionary(nx, ny, (2, 3), (0.0, 90.0, 45.0))
    x = orc.pixel_positions(nx, ny, 1.0)
    f = orc.frequencies(7, 9.9e9, 10.1e9)
    rng = np.random.default_rng(9)
    p_n = np.zeros((nx * ny, nx * ny), dtype=np.complex128)
    b_pix = np.zeros(nx * ny, dtype=np.complex128)
    g_n = np.zeros((h.shape[1], h.shape[1]), dtype=np.complex128)
    b_n = np.zeros(h.shape[1], dtype=np.complex128)
    for k in range(3):
        gamma = np.array([900.0 * np.cos(0.1 * k), 900.0 * np.sin(0.1 * k), 400.0])
        fs = orc.phase_matrix(gamma, x, f)
        d = rng.standard_normal(7) + 1j * rng.standard_normal(7)
        p_n += orc.gram_increment(orc.forward_block(fs, None))
        b_pix += orc.data_increment(orc.forward_block(fs, None), d)
        a_s = orc.forward_block(fs, h)
        g_n += orc.gram_increment(a_s)
        b_n += orc.data_increment(a_s, d)
    assert np.allclose(h.conj().T @ p_n @ h, g_n, rtol=0, atol=1e-10 * np.abs(g_n).max())
    assert np.allclose(h.conj().T @ b_pix, b_n, rtol=0, atol=1e-12 * np.abs(b_n).max())
    # applied as three steps on a vector: u = H x, w = P u, H^H w
    c = rng.standard_normal(h.shape[1]) + 1j * rng.standard_normal(h.shape[1])
    u = np.array([c[h[p] != 0].sum() for p in range(nx * ny)])
    w = p_n @ u
    y = np.array([w[h[:, m] != 0].sum() for m in range(h.shape[1])])
    assert np.allclose(y, g_n @ c, rtol=0, atol=1e-10 * np.abs(g_n @ c).max())


def test_non_white_increments_are_the_weighted_sums():
    # Eq. 12 with R_n = diag(var): entrywise sums with weights 1 / var_k, and
    # a constant variance scales the white increments
    rng = np.random.default_rng(5)
    a = rng.standard_normal((6, 4)) + 1j * rng.standard_normal((6, 4))
    d = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    var = rng.uniform(0.5, 3.0, 6)
    g = orc.gram_increment(a, var)
    for i in range(4):
        for j in range(4):
            want = sum(np.conj(a[k, i]) * a[k, j] / var[k] for k in range(6))
            assert abs(g[i, j] - want) <= 1e-12 * max(1.0, abs(want))
    b = orc.data_increment(a, d, var)
    assert np.allclose(b, [sum(np.conj(a[k, i]) * d[k] / var[k] for k in range(6))
                           for i in range(4)], rtol=1e-13, atol=0)
    assert np.allclose(orc.gram_increment(a, np.full(6, 4.0)),
                       orc.gram_increment(a) / 4.0, rtol=1e-13, atol=0)


# ------------------------------------------------- the online trajectory ---

@pytest.mark.parametrize("dictionary", [None, "gaussian"])
def test_online_trajectory_pulse_by_pulse(dictionary):
    """The online run pinned pulse by pulse to what the paper fixes, so that
    a mistake anywhere along the trajectory (lambda's schedule, the Lipschitz
    bound, the warm start, the carried momentum, the problem each burst
    solves) fails here and not only in oracle-GPU agreement:

    * lambda_n = rho max|b_n| with b_n the batch sum over the pulses so far,
      formed here from the phase matrices with an einsum (Eqs. 11, 13);
    * L_n is non-decreasing, at most (1 + delta) lambda_max(G_n), and where
      it grew it is (1 + delta) times the last power step's Rayleigh
      quotient, hence at most that of the stored power vector (one more step
      on a PSD matrix can only raise it) (Eq. 14, Eq. 11);
    * a burst starts from the previous pulse's image (c^(0) = z^(1) =
      c_hat_{n-1}) with t carried (t_1 = 1 only on the first pulse);
    * run to convergence, every pulse's image satisfies the LASSO
      optimality conditions of (G_n, b_n, lambda_n) (Eq. 8)."""
    if dictionary is None:
        w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=6, seed=4)
    else:
        w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=6, seed=4,
                           dictionary="gaussian", n_atoms=50, dict_seed=3)
    track, dic, _, data = build_problem(w)
    cfg = oracle_config(w, dic, lam=0.05)
    of = orc.OnlineFista(cfg)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    blocks = []
    lip_prev = 0.0
    c_prev_pulse = np.zeros(of.m, complex)
    t_prev = None
    for n in range(w.n_pulses):
        of.push_pulse(track[n], data[n])
        p = orc.phase_matrix(track[n], x, f)
        blocks.append(p if dic is None else p @ dic)
        a = np.stack(blocks)                          # pulses x K x M
        b_batch = np.einsum("skm,sk->m", a.conj(), data[: n + 1])
        g_batch = np.einsum("skm,skj->mj", a.conj(), a)
        s = of.s
        assert abs(s.lam - 0.05 * np.max(np.abs(b_batch))) <= 1e-12 * s.lam
        eig = np.linalg.eigvalsh(g_batch)
        mu = float(np.real(np.vdot(s.v, g_batch @ s.v)) / np.vdot(s.v, s.v).real)
        assert s.lip >= lip_prev
        assert s.lip <= (1 + cfg.lipschitz_margin) * eig[-1] * (1 + 1e-12)
        if s.lip > lip_prev:
            assert s.lip <= (1 + cfg.lipschitz_margin) * mu * (1 + 1e-12)
        lip_prev = s.lip
        assert of.iterate(0) == 0                      # starts the burst only
        assert np.array_equal(s.z, c_prev_pulse)
        assert np.array_equal(s.c_prev, c_prev_pulse)
        assert s.t == (1.0 if n == 0 else t_prev)
        of.iterate(200000, 1e-13)
        assert orc.kkt_residual(g_batch, b_batch, s.c_hat, s.lam) <= 1e-6, n
        c_prev_pulse = s.c_hat.copy()
        t_prev = s.t
