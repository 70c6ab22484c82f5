"""Failure detection without a GPU fault: every wait inside the kernels is
bounded by the GPU clock, and a wait that runs out records a timeout in the
context's device error word, stops its CTA and returns.  The check drives
that path with a barrier nothing ever completes (osar_probe_bounded_wait) and
verifies the status the host reads, the time it took, and that the GPU
serves the next context as before.  Host-side failures (invalid arguments,
calls in the wrong state) are covered in test_abi_cpu.py and
test_gpu_parity.py."""
import time

import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import (small_workload, build_problem, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config, run_pair

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_gpu_stays_usable():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=3, seed=7)
    g = osar.Osar(gpu_config(w, "split_bf16"))
    t0 = time.perf_counter()
    st = g.probe_bounded_wait(50_000_000)          # 50 ms
    dt = time.perf_counter() - t0
    assert st == osar.OSAR_E_TIMEOUT
    assert 0.04 <= dt < 5.0
    # the recorded timeout is reported by the context's next state read
    with pytest.raises(osar.OsarError) as e:
        g.state()
    assert e.value.status == osar.OSAR_E_TIMEOUT
    g.close()
    # a new context on the same GPU runs the path and meets its parity bar
    of, g2 = run_pair(w, "split_bf16", steps=8)
    assert_coeffs(g2.coeffs(), of.s, 1e-3, SUPPORT_DELTA["split_bf16"])


def test_bounded_wait_rejects_out_of_range_limits():
    w = small_workload(nx=8, ny=8, n_freq=16, n_pulses=1, seed=7)
    g = osar.Osar(gpu_config(w, "fp64"))
    assert g.probe_bounded_wait(10) == osar.OSAR_E_INVALID
    assert g.probe_bounded_wait(10**12) == osar.OSAR_E_INVALID
    g.state()                                      # nothing recorded
