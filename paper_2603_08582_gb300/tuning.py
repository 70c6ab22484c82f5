"""Online lambda tuning driven by the library's adjoint (osar_unroll_grad).

The paper leaves online parameter tuning to future work (Sec. I, Sec. V).
This module is the library's rule for it.  Every `every` pulses, after the
pulse is pushed and before its burst runs, the burst is differentiated: with
c_T(lambda) the result of T steps of Algorithm 1 from c_hat_{n-1} on the
pulse's statistics (A_n, b_n), its step tau = 1/L_n and momentum t, and the
loss L = ||c_T - c_ref||^2 against a reference scene (a calibration target;
the synthetic truth in the benchmark), the adjoint kernels give dL/dlambda.
The relative setting rho (lambda_n = rho ||b_n||_inf) then takes a
normalised step in log space,

    log rho <- log rho - eta * clip(lambda_n dL/dlambda / L, -1, 1),

and osar_set_lambda applies it from the next pulse.  Only the step rule runs
on the host; the gradient is the library's (every Gram pass on the device).
"""
from __future__ import annotations

import math

import numpy as np


def lambda_update(rho: float, lam: float, d_lam: float, loss: float,
                  eta: float) -> float:
    """One step of the rule above: the loss's relative sensitivity to
    log lambda, clipped to [-1, 1], scaled by eta, taken against its sign."""
    if not (loss > 0.0) or not math.isfinite(d_lam) or lam <= 0.0:
        return rho
    g = max(-1.0, min(1.0, lam * d_lam / loss))
    return rho * math.exp(-eta * g)


class OnlineLambdaTuner:
    """Tunes a relative-lambda context's factor rho while pulses arrive.

    ctx: an osar.Osar with lambda_relative; c_ref: the reference
    coefficients (M complex); steps: the burst length T the gradient
    unrolls; every: pulses between updates; eta: the log-space step."""

    def __init__(self, ctx, c_ref, rho: float, steps: int, every: int = 8,
                 eta: float = 0.25, ckpt_every: int | None = None,
                 restart_momentum: bool = False):
        self.ctx = ctx
        self.c_ref = np.ascontiguousarray(np.asarray(c_ref, dtype=np.complex128))
        self.rho = float(rho)
        self.steps = int(steps)
        self.every = max(1, int(every))
        self.eta = float(eta)
        self.ckpt = ckpt_every or max(1, int(round(math.sqrt(self.steps))))
        self.restart = restart_momentum
        self.history = []
        ctx.set_lambda(self.rho)

    def after_push(self, pulse: int):
        """Call after pushing pulse `pulse` (0-based), before its burst."""
        if pulse % self.every:
            return None
        st = self.ctx.state()
        if st["lipschitz"] <= 0.0 or st["lambda"] <= 0.0:
            return None
        c0 = self.ctx.coeffs()                      # c_hat_{n-1}
        t0 = 1.0 if (st["n"] == 1 or self.restart) else st["t"]
        g = self.ctx.unroll_grad(self.steps, self.ckpt, st["lambda"],
                                 1.0 / st["lipschitz"], c0, self.c_ref, t0=t0)
        rho = lambda_update(self.rho, st["lambda"], g["d_lambda"], g["loss"],
                            self.eta)
        rec = {"pulse": pulse, "rho": self.rho, "lambda": st["lambda"],
               "loss": g["loss"], "d_lambda": g["d_lambda"], "rho_next": rho}
        self.history.append(rec)
        if rho != self.rho:
            self.rho = rho
            self.ctx.set_lambda(rho)
        return rec
