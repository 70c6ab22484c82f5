"""CTA-pair tensor-core products (tc_pairs = 1: one M = 256 tcgen05 MMA on
two SMs per two Gram or dictionary blocks that share their B rows) against
one SM per block (tc_pairs = 0): the same MMA order per entry, so the same
bits, for dictionary and pixel-basis models, odd block counts (a pair with a
missing second block), and a capped dictionary grid (one pair)."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _run(w, problem, pairs, synth_ctas=0, steps=10):
    cfg = gpu_config(w, "split_bf16")
    cfg.tc_pairs = 3 if pairs else 0  # both products on SM pairs, or neither
    # the power step fused into the pair kernel's Gram update sums in another
    # order than a separate pass; compare like with like
    cfg.fuse_power_gram = 0
    cfg.synth_ctas = int(synth_ctas)
    g = osar.Osar(cfg)
    track, _, _, data = problem
    for s in range(track.shape[0]):
        g.push_pulse(track[s], data[s])
        g.iterate(steps, 0.0, want_count=False)
    g.synchronize()
    return g


def _same(a, b):
    ga, gb = a.gram(), b.gram()
    assert np.array_equal(ga, gb), np.max(np.abs(ga - gb)) / np.max(np.abs(ga))
    assert np.array_equal(a.coeffs(), b.coeffs())
    assert a.state() == b.state()


@pytest.mark.parametrize("synth_ctas", [0, 2])
def test_pairs_match_single_sm_dictionary(synth_ctas):
    # 24 x 24 pixels, M = 1100 atoms: 9 atom blocks (odd), K = 96
    w = small_workload(nx=24, ny=24, n_freq=96, n_pulses=5,
                       dictionary="gaussian", n_atoms=1100, sparsity=0.03,
                       seed=31, dict_seed=6)
    problem = build_problem(w)
    _same(_run(w, problem, False), _run(w, problem, True, synth_ctas))


def test_pairs_match_single_sm_pixel_basis():
    # 40 x 40 pixel basis: M = 1600, 13 blocks (odd)
    w = small_workload(nx=40, ny=40, n_freq=128, n_pulses=4, sparsity=0.03,
                       seed=32)
    problem = build_problem(w)
    _same(_run(w, problem, False), _run(w, problem, True))
