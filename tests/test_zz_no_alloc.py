"""The allocation-free Gram apply, osar_gram_apply_static.

Callers that must not allocate device memory once they are running (fixed
memory budgets on embedded or flight systems, hosts that hand out every
buffer from their own pool) use this entry point: they pass x and y in
device memory and the matvec's scratch comes from a static array inside the
library.  These tests check it against the allocating entry point,
osar_gram_apply, on two calls in a row (the shared array keeps the previous
call's contents), and check the clear rejection above its size limit.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar, synth
from tests.helpers import small_workload, build_problem, rel_err
from tests.gpu_helpers import gpu_config

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "split_bf16": 1e-4}


def _context(prec):
    w = small_workload(nx=32, ny=32, n_freq=48, n_pulses=5, seed=17)
    track, dic, c_true, data = build_problem(w)
    g = osar.Osar(gpu_config(w, prec))
    for s in range(w.n_pulses):
        g.push_pulse(track[s], data[s])
        g.iterate(3)
    return w, g


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_static_apply_matches_allocating_apply_twice(prec):
    w, g = _context(prec)
    rng = np.random.default_rng(5)
    for _ in range(2):
        x = (rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms))
        y_ref = g.gram_apply(x)
        x_dev = torch.from_numpy(x).to("cuda")
        y_dev = torch.full((w.m_atoms,), complex(np.nan, np.nan),
                           dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
        g.synchronize()
        y = y_dev.cpu().numpy()
        assert np.all(np.isfinite(y))
        assert rel_err(y, y_ref) <= TOL[prec]


def test_static_apply_rejects_gram_beyond_static_scratch():
    w = small_workload(nx=128, ny=64, n_freq=16, n_pulses=1)
    g = osar.Osar(gpu_config(w, "fp32"))
    x_dev = torch.zeros(w.m_atoms, dtype=torch.complex128, device="cuda")
    y_dev = torch.zeros_like(x_dev)
    with pytest.raises(osar.OsarError) as ei:
        g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
    assert ei.value.status == osar.OSAR_E_INVALID
    assert "static" in str(ei.value)
