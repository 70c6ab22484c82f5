"""Guard regions (guard_bytes) as a memory check without compute-sanitizer:
every device buffer of a context or a batch is followed by bytes of a known
fill, and no kernel of any form may change them.  Each case runs a form with
guards on and checks that no guard changed; a guard overwritten on purpose
from the host must be found and named."""
import os

import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

GUARD = 4096


def _cfg(w, prec, **kw):
    cfg = gpu_config(w, prec, **kw)
    cfg.guard_bytes = GUARD
    return cfg


def _pulses(g, w, steps=8, tol=0.0, pulses=None):
    track, _, c_true, data = build_problem(w)
    for s in range(track.shape[0] if pulses is None else pulses):
        g.push_pulse(track[s], data[s])
        g.iterate(steps, tol, want_count=False)
    return track, c_true


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_pixel_basis_readbacks_and_checkpoint_leave_guards(prec, tmp_path):
    # 20 x 20 pixels (M = 400, 4 blocks, ragged), K = 36 (ragged)
    w = small_workload(nx=20, ny=20, n_freq=36, n_pulses=5, sparsity=0.05, seed=31)
    g = osar.Osar(_cfg(w, prec))
    track, c_true = _pulses(g, w, steps=10, tol=1e-6)
    g.gram()
    g.b()
    g.gram_apply(np.ones(w.m_atoms, complex))
    g.simulate_pulse(track[0], c_true)
    path = os.path.join(tmp_path, "ck.bin")
    g.save(path)
    assert g.check_guards() == 0
    h = osar.Osar.load(path, _cfg(w, prec))
    _pulses(h, w, steps=4, pulses=2)
    assert h.check_guards() == 0


@pytest.mark.parametrize("defer", [False, True])
def test_dictionary_overlap_and_deferred_update_leave_guards(defer):
    w = small_workload(nx=24, ny=24, n_freq=96, n_pulses=6, dictionary="gaussian",
                       n_atoms=1100, sparsity=0.03, seed=21, dict_seed=4)
    g = osar.Osar(_cfg(w, "split_bf16", defer_gram=defer))
    _pulses(g, w, steps=12, tol=1e-5)
    g.gram()
    assert g.check_guards() == 0


def test_lambda_path_and_adjoint_leave_guards():
    w = small_workload(nx=16, ny=16, n_freq=48, n_pulses=4, dictionary="gaussian",
                       n_atoms=300, sparsity=0.04, seed=42, dict_seed=3)
    cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                           pixel_m=w.pixel_m, precision="split_bf16",
                           dictionary="gaussian", n_atoms=w.m_atoms,
                           dict_seed=w.dict_seed, lambdas=[0.03, 0.05, 0.08],
                           guard_bytes=GUARD)
    g = osar.Osar(cfg)
    _pulses(g, w, steps=10)
    for l in range(3):
        g.lambda_state(l)
    assert g.check_guards() == 0
    for prec in ("fp64", "fp32"):
        a = osar.Osar(_cfg(w, prec))
        _, c_true = _pulses(a, w, steps=6)
        st = a.state()
        a.unroll_grad(16, 4, st["lambda"], 1.0 / st["lipschitz"], a.coeffs(), c_true)
        assert a.check_guards() == 0


def test_batch_leaves_guards():
    ws = [small_workload(nx=nx, ny=ny, n_freq=k, n_pulses=4, seed=100 + i)
          for i, (nx, ny, k) in enumerate([(8, 8, 16), (12, 12, 24), (9, 13, 28)])]
    cfgs = [_cfg(w, "split_bf16") for w in ws]
    b = osar.OsarBatch(cfgs)
    probs = [build_problem(w) for w in ws]
    for s in range(4):
        gam = np.stack([p[0][s] for p in probs])
        b.push([1, 1, 1], gam, [p[3][s] for p in probs])
        b.iterate(6, 1e-6)
    assert b.check_guards() == 0


def test_an_overwritten_guard_is_found_and_named():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=2, seed=7)
    g = osar.Osar(_cfg(w, "fp32"))
    _pulses(g, w, steps=4)
    assert g.check_guards() == 0
    assert g.poke_guard(2) == osar.OSAR_OK
    assert g.check_guards() == 1
    assert "guard overwritten behind" in g.last_error()
    assert g.poke_guard(10**6) == osar.OSAR_E_INVALID
