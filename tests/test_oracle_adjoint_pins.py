"""Pins for the FP64 autograd reference of the unrolled FISTA map: central
finite differences (h = 1e-6) in float64, and the d-gradient chain rule
through b = sum_s G_s^H d_s checked against finite differences in d."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import osar_oracle as orc
from oracle import adjoint_oracle as adj
from tests.helpers import small_workload, build_problem, oracle_config


def _setup(seed=0, steps=24):
    w = small_workload(nx=6, ny=6, n_freq=12, n_pulses=6, seed=seed)
    track, dic, c_true, data = build_problem(w)
    of = orc.OnlineFista(oracle_config(w, None))
    blocks = []
    for s in range(w.n_pulses):
        of.push_pulse(track[s], data[s])
        blocks.append(of.block(track[s]))
    g, b = of.s.gram, of.s.b
    lam = of.s.lam
    tau = 1.0 / of.s.lip
    c0 = np.zeros_like(b)
    return g, b, c0, lam, tau, c_true, steps, blocks, data


def _margin_ok(g, b, c0, lam, tau, steps, h):
    """Reject kinks: no |u_k| within a relative 100 h of lambda tau."""
    c_prev = c0.copy()
    z = c0.copy()
    t = 1.0
    for _ in range(steps):
        u = z - tau * (g @ z - b)
        if np.min(np.abs(np.abs(u) - lam * tau)) < 100 * h * lam * tau:
            return False
        c = orc.soft_threshold(u, lam * tau)
        tn = orc.momentum_next(t)
        z = c + ((t - 1) / tn) * (c - c_prev)
        c_prev, t = c, tn
    return True


@pytest.mark.parametrize("seed", [0, 3])
def test_autograd_matches_central_differences(seed):
    g, b, c0, lam, tau, c_true, steps, blocks, data = _setup(seed)
    h = 1e-6
    assert _margin_ok(g, b, c0, lam, tau, steps, h)
    ref = adj.gradients(g, b, c0, lam, tau, c_true, steps, blocks=blocks)
    f = lambda l, t_, bb: adj.loss_value(g, bb, c0, l, t_, c_true, steps)
    # lambda and tau: relative steps
    hl = h * lam
    fd_l = (f(lam + hl, tau, b) - f(lam - hl, tau, b)) / (2 * hl)
    ht = h * tau
    fd_t = (f(lam, tau + ht, b) - f(lam, tau - ht, b)) / (2 * ht)
    assert abs(fd_l - ref["d_lambda"]) <= 1e-5 * abs(fd_l)
    assert abs(fd_t - ref["d_tau"]) <= 1e-5 * abs(fd_t)
    # data: Re and Im of a few entries of a few pulses
    rng = np.random.default_rng(seed)
    for _ in range(4):
        s = int(rng.integers(0, len(data)))
        k = int(rng.integers(0, data.shape[1]))
        for unit in (1.0, 1j):
            hd = h * np.max(np.abs(data))
            dp = data.copy()
            dm = data.copy()
            dp[s, k] += unit * hd
            dm[s, k] -= unit * hd
            bp = orc.batch_data(blocks, list(dp))
            bm = orc.batch_data(blocks, list(dm))
            fd = (f(lam, tau, bp) - f(lam, tau, bm)) / (2 * hd)
            got = ref["d_data"][s][k]
            comp = got.real if unit == 1.0 else got.imag
            assert abs(fd - comp) <= 1e-4 * max(abs(fd), 1e-3 * np.max(np.abs(ref["d_data"][s])))


def test_complex_gradient_convention():
    """torch reports dL/dRe + i dL/dIm for a real loss of a complex input."""
    z = torch.tensor([1.0 + 2.0j], dtype=torch.complex128, requires_grad=True)
    loss = torch.real(z * z.conj()).sum() + 3.0 * torch.imag(z).sum()
    loss.backward()
    # L = x^2 + y^2 + 3y  =>  dL/dx = 2, dL/dy = 4 + 3 = 7
    assert complex(z.grad[0]) == pytest.approx(2.0 + 7.0j)
