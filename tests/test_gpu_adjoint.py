"""GPU checks of the differentiation form (osar_unroll_grad and the
torch.autograd.Function on top of it) against the FP64 autograd oracle and
central finite differences (h = 1e-6).

Tolerances: FP64 adjoint vs FP64 autograd <= 1e-8 relative; FP32-Gram
adjoint vs FP64 <= 1e-4; finite differences vs the FP64 adjoint <= 1e-4
(the required bar).  Coordinates within 100 h of the shrinkage kink
|u| = lambda tau would make differences meaningless, so the tests check the
recorded margin first and nudge lambda until it is clear.

Conditioning of dL/dtau.  After many unrolled steps c_T is close to the
LASSO solution, which depends on lambda but not on tau, so dL/dtau is the
small difference of two large terms (the step term and lambda dL/dalpha);
on the 64 x 64 workload tau |dL/dtau| / L ~ 1e-6.  Two consequences, both
measured on GB300: a central difference with h = 1e-6 (relative) resolves
dL/dtau only to ~3e-4 even in FP64 (rounding of L divided by 2 h tau), so
the tau check uses h = 1e-5; and an FP32-Gram trajectory (relative error
~1e-7) cannot resolve dL/dtau itself, so the FP32 tau-gradient is compared
with the FP64 one relative to the size of the cancelling terms,
lambda |dL/dlambda| / tau.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import osar_oracle as orc
from oracle import adjoint_oracle as adj
from paper_2603_08582_gb300 import osar, synth
from paper_2603_08582_gb300.autograd import unrolled_loss
from tests.helpers import small_workload, build_problem, oracle_config, rel_err
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

H = 1e-6


def _kink_margin(g, b, c0, lam, tau, steps):
    """min over steps and coordinates of ||u| - lambda tau| / (lambda tau)."""
    c_prev = c0.copy()
    z = c0.copy()
    t = 1.0
    worst = np.inf
    for _ in range(steps):
        u = z - tau * (g @ z - b)
        worst = min(worst, float(np.min(np.abs(np.abs(u) - lam * tau))) / (lam * tau))
        c = orc.soft_threshold(u, lam * tau)
        tn = orc.momentum_next(t)
        z = c + ((t - 1) / tn) * (c - c_prev)
        c_prev, t = c, tn
    return worst


def _setup(w, precs, steps):
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, dic))
    ctxs = {p: osar.Osar(gpu_config(w, p)) for p in precs}
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
        for c in ctxs.values():
            c.push_pulse(track[s], data[s])
    g, b = of.s.gram, of.s.b
    lam = of.s.lam
    tau = 1.0 / of.s.lip
    c0 = np.zeros_like(b)
    for _ in range(20):
        if _kink_margin(g, b, c0, lam, tau, steps) > 100 * H:
            break
        lam *= 1.0007
    return track, data, c_true, of, ctxs, g, b, lam, tau, c0


def test_adjoint_matches_autograd_and_differences_small():
    w = small_workload(nx=12, ny=12, n_freq=24, n_pulses=8, sparsity=0.05, seed=31)
    steps, ckpt = 16, 4
    track, data, c_true, of, ctxs, g, b, lam, tau, c0 = _setup(
        w, ("fp64", "fp32", "split_bf16"), steps)
    ref = adj.gradients(g, b, c0, lam, tau, c_true, steps)
    r64 = ctxs["fp64"].unroll_grad(steps, ckpt, lam, tau, c0, c_true)
    assert abs(r64["loss"] - ref["loss"]) <= 1e-9 * ref["loss"]
    assert abs(r64["d_lambda"] - ref["d_lambda"]) <= 1e-8 * abs(ref["d_lambda"])
    assert abs(r64["d_tau"] - ref["d_tau"]) <= 1e-8 * abs(ref["d_tau"])
    assert rel_err(r64["d_b"], ref["d_b"]) <= 1e-8
    assert rel_err(r64["c_T"], adj.unrolled_forward(g, b, c0, lam, tau, steps)) <= 1e-9
    for p in ("fp32", "split_bf16"):
        r = ctxs[p].unroll_grad(steps, ckpt, lam, tau, c0, c_true)
        assert abs(r["d_lambda"] - r64["d_lambda"]) <= 1e-4 * abs(r64["d_lambda"]), p
        assert abs(r["d_tau"] - r64["d_tau"]) <= 1e-4 * abs(r64["d_tau"]), p
        assert rel_err(r["d_b"], r64["d_b"]) <= 1e-4, p
    # central differences of the GPU's own FP64 loss
    gp = ctxs["fp64"]
    f = lambda l, t: gp.unroll_grad(steps, ckpt, l, t, c0, c_true)["loss"]
    fd_l = (f(lam * (1 + H), tau) - f(lam * (1 - H), tau)) / (2 * H * lam)
    fd_t = (f(lam, tau * (1 + H)) - f(lam, tau * (1 - H))) / (2 * H * tau)
    assert abs(fd_l - r64["d_lambda"]) <= 1e-4 * abs(fd_l)
    assert abs(fd_t - r64["d_tau"]) <= 1e-4 * abs(fd_t)


def test_checkpoint_interval_does_not_change_gradients():
    w = small_workload(nx=10, ny=10, n_freq=20, n_pulses=6, seed=5)
    track, data, c_true, of, ctxs, g, b, lam, tau, c0 = _setup(w, ("fp64",), 13)
    gp = ctxs["fp64"]
    a = gp.unroll_grad(13, 1, lam, tau, c0, c_true)
    for ck in (3, 5, 13, 40):
        r = gp.unroll_grad(13, ck, lam, tau, c0, c_true)
        assert r["loss"] == a["loss"]
        assert r["d_lambda"] == a["d_lambda"] and r["d_tau"] == a["d_tau"]
        assert np.array_equal(r["d_b"], a["d_b"])


def test_data_gradient_and_autograd_function():
    w = small_workload(nx=10, ny=10, n_freq=20, n_pulses=5, seed=11)
    steps = 12
    track, data, c_true, of, ctxs, g, b, lam, tau, c0 = _setup(w, ("fp64",), steps)
    gp = ctxs["fp64"]
    blocks = [of.block(gm) for gm in track]
    ref = adj.gradients(g, b, c0, lam, tau, c_true, steps, blocks=blocks)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    tau_t = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
    d_t = torch.from_numpy(data.copy()).requires_grad_(True)
    loss = unrolled_loss(gp, lam_t, tau_t, d_t, track, c0, c_true, steps)
    (3.0 * loss).backward()
    assert abs(loss.item() - ref["loss"]) <= 1e-9 * ref["loss"]
    assert abs(lam_t.grad.item() - 3 * ref["d_lambda"]) <= 1e-8 * abs(3 * ref["d_lambda"])
    assert abs(tau_t.grad.item() - 3 * ref["d_tau"]) <= 1e-8 * abs(3 * ref["d_tau"])
    dd_ref = 3 * np.stack(ref["d_data"])
    assert rel_err(d_t.grad.numpy(), dd_ref) <= 1e-8
    # one data entry by central differences through fresh contexts
    s, k = 2, 7
    hd = H * np.max(np.abs(data))

    def loss_with(dd):
        c = osar.Osar(gpu_config(w, "fp64"))
        for q in range(w.n_pulses):
            c.push_pulse(track[q], dd[q])
        return c.unroll_grad(steps, 4, lam, tau, c0, c_true)["loss"]

    for unit in (1.0, 1j):
        dp, dm = data.copy(), data.copy()
        dp[s, k] += unit * hd
        dm[s, k] -= unit * hd
        fd = (loss_with(dp) - loss_with(dm)) / (2 * hd)
        got = dd_ref[s, k] / 3
        comp = got.real if unit == 1.0 else got.imag
        assert abs(fd - comp) <= 1e-4 * max(abs(fd), 1e-3 * np.max(np.abs(dd_ref)))


def test_adjoint_64x64_full_config():
    """The 64 x 64 / K = 256 / 128-pulse workload, T = 64 unrolled steps with
    sqrt(T) = 8 checkpoints: FP64 adjoint vs the FP64 autograd oracle and
    central differences; FP32 adjoint vs FP64."""
    w = synth.workloads()["c3_64x64_adjoint"]
    steps, ckpt = w.extra["unroll_T"], w.extra["checkpoint_every"]
    track, data, c_true, of, ctxs, g, b, lam, tau, c0 = _setup(
        w, ("fp64", "fp32"), steps)
    ref = adj.gradients(g, b, c0, lam, tau, c_true, steps)
    r64 = ctxs["fp64"].unroll_grad(steps, ckpt, lam, tau, c0, c_true)
    r32 = ctxs["fp32"].unroll_grad(steps, ckpt, lam, tau, c0, c_true)
    print("c3 adjoint:", r64["d_lambda"], ref["d_lambda"], r32["d_lambda"])
    assert abs(r64["d_lambda"] - ref["d_lambda"]) <= 1e-7 * abs(ref["d_lambda"])
    assert abs(r64["d_tau"] - ref["d_tau"]) <= 1e-7 * abs(ref["d_tau"])
    assert rel_err(r64["d_b"], ref["d_b"]) <= 1e-7
    assert abs(r32["d_lambda"] - r64["d_lambda"]) <= 1e-4 * abs(r64["d_lambda"])
    assert rel_err(r32["d_b"], r64["d_b"]) <= 1e-4
    scale_tau = lam * abs(r64["d_lambda"]) / tau      # size of the cancelling terms
    assert abs(r32["d_tau"] - r64["d_tau"]) <= 1e-4 * scale_tau
    gp = ctxs["fp64"]
    f = lambda l, t: gp.unroll_grad(steps, ckpt, l, t, c0, c_true)["loss"]
    fd_l = (f(lam * (1 + H), tau) - f(lam * (1 - H), tau)) / (2 * H * lam)
    ht = 10 * H
    fd_t = (f(lam, tau * (1 + ht)) - f(lam, tau * (1 - ht))) / (2 * ht * tau)
    assert abs(fd_l - r64["d_lambda"]) <= 1e-4 * abs(fd_l)
    assert abs(fd_t - r64["d_tau"]) <= 1e-4 * abs(fd_t)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_replayed_gradient_sequence_takes_new_arguments(prec):
    """The gradient's device sequence is captured once per (T, checkpoint
    interval) and replayed: a replay with other lambda, tau, t0, c0 and
    c_true, and a call with another T (a new capture) in between, give
    bitwise what a fresh context computes for the same call."""
    w = small_workload(nx=10, ny=10, n_freq=20, n_pulses=5, sparsity=0.06, seed=37)
    track, _, c_true, data = build_problem(w)
    a = osar.Osar(gpu_config(w, prec))
    for s in range(w.n_pulses):
        a.push_pulse(track[s], data[s])
    st = a.state()
    lam, tau = st["lambda"], 1.0 / st["lipschitz"]
    rng = np.random.default_rng(3)
    c0 = 0.1 * (rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms))
    calls = [(12, 3, lam, tau, 1.0, np.zeros(w.m_atoms, complex), c_true),
             (12, 3, 1.3 * lam, 0.9 * tau, 2.5, c0, 0.5 * c_true),
             (7, 2, 0.8 * lam, tau, 1.0, c0, c_true),
             (12, 3, 0.7 * lam, 0.95 * tau, 1.7, -c0, c_true)]
    for T, C, l, t, t0, x0, ct in calls:
        got = a.unroll_grad(T, C, l, t, x0, ct, t0=t0)
        b = osar.Osar(gpu_config(w, prec))
        for s in range(w.n_pulses):
            b.push_pulse(track[s], data[s])
        want = b.unroll_grad(T, C, l, t, x0, ct, t0=t0)
        b.close()
        for k in ("loss", "d_lambda", "d_tau"):
            assert got[k] == want[k], (T, k)
        assert np.array_equal(got["d_b"], want["d_b"])
        assert np.array_equal(got["c_T"], want["c_T"])
