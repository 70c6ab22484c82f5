"""FP64 autograd reference for the differentiation form of Online FISTA.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU-baseline
leg, never by the product path.  Plain PyTorch CPU ops in float64 /
complex128; gradients come from torch.autograd, and the tests pin them with
central finite differences.

The unrolled map (Algorithm 1's inner loop on a fixed Gram G and data vector
b, §III-C): z_1 = c_0, t_1 = t0, and for k = 1..T

    u_k = z_k - tau (G z_k - b)
    c_k = S_{lambda tau}(u_k)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    z_{k+1} = c_k + (t_k - 1) / t_{k+1} (c_k - c_{k-1})

with loss ||c_T - c_true||_2^2.  The data vector is b = sum_s G_s^H d_s
(Eqs. 12-13), so gradients with respect to the pulse data d_s follow from
the gradient with respect to b.  Complex gradients use the convention
dL/dRe + i dL/dIm (what torch reports for a real loss).
"""
from __future__ import annotations

import numpy as np
import torch


def _shrink(u: torch.Tensor, alpha: torch.Tensor) -> torch.Tensor:
    """Complex shrinkage u max(0, 1 - alpha/|u|), exactly 0 where |u| <= alpha."""
    mag = torch.abs(u)
    keep = mag > alpha
    safe = torch.where(keep, mag, torch.ones_like(mag))
    scale = torch.where(keep, 1.0 - alpha / safe, torch.zeros_like(mag))
    return u * scale


def unrolled_loss(g: torch.Tensor, b: torch.Tensor, c0: torch.Tensor,
                  lam: torch.Tensor, tau: torch.Tensor, c_true: torch.Tensor,
                  steps: int, t0: float = 1.0) -> torch.Tensor:
    c_prev = c0
    z = c0
    t = t0
    for _ in range(steps):
        u = z - tau * (g @ z - b)
        c = _shrink(u, lam * tau)
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = c + ((t - 1.0) / t_next) * (c - c_prev)
        c_prev = c
        t = t_next
    r = c_prev - c_true
    return torch.sum(torch.real(r) ** 2 + torch.imag(r) ** 2)


def unrolled_forward(g, b, c0, lam: float, tau: float, steps: int,
                     t0: float = 1.0) -> np.ndarray:
    """c_T of the unrolled map, NumPy in / NumPy out."""
    with torch.no_grad():
        gt = torch.as_tensor(np.asarray(g, dtype=np.complex128))
        bt = torch.as_tensor(np.asarray(b, dtype=np.complex128))
        c_prev = torch.as_tensor(np.asarray(c0, dtype=np.complex128))
        z = c_prev
        t = t0
        lam_t = torch.tensor(lam, dtype=torch.float64)
        tau_t = torch.tensor(tau, dtype=torch.float64)
        for _ in range(steps):
            u = z - tau_t * (gt @ z - bt)
            c = _shrink(u, lam_t * tau_t)
            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            z = c + ((t - 1.0) / t_next) * (c - c_prev)
            c_prev = c
            t = t_next
        return c_prev.numpy()


def gradients(g, b, c0, lam: float, tau: float, c_true, steps: int,
              t0: float = 1.0, blocks=None):
    """Loss and its gradients with respect to lambda, tau and b (and, when the
    per-pulse blocks G_s are given, the pulse data d_s through b)."""
    gt = torch.as_tensor(np.asarray(g, dtype=np.complex128))
    bt = torch.as_tensor(np.asarray(b, dtype=np.complex128)).clone().requires_grad_(True)
    c0t = torch.as_tensor(np.asarray(c0, dtype=np.complex128))
    ctt = torch.as_tensor(np.asarray(c_true, dtype=np.complex128))
    lam_t = torch.tensor(float(lam), dtype=torch.float64, requires_grad=True)
    tau_t = torch.tensor(float(tau), dtype=torch.float64, requires_grad=True)
    loss = unrolled_loss(gt, bt, c0t, lam_t, tau_t, ctt, steps, t0)
    loss.backward()
    out = {
        "loss": float(loss.detach()),
        "d_lambda": float(lam_t.grad),
        "d_tau": float(tau_t.grad),
        "d_b": bt.grad.numpy().copy(),
    }
    if blocks is not None:
        # b = sum_s G_s^H d_s  =>  dL/dd_s = G_s dL/db (same convention)
        out["d_data"] = [np.asarray(a) @ out["d_b"] for a in blocks]
    return out


def loss_value(g, b, c0, lam: float, tau: float, c_true, steps: int,
               t0: float = 1.0) -> float:
    c = unrolled_forward(g, b, c0, lam, tau, steps, t0)
    r = c - np.asarray(c_true)
    return float(np.sum(np.abs(r) ** 2))
