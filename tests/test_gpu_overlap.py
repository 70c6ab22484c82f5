"""Overlapped synthesis: the phase synthesis and dictionary product of a
pushed pulse run on a side stream beside the previous pulse's burst.  Every
result must stay bitwise the same as with the overlap off, for automatic and
capped dictionary grids, pulses from host or device memory, no host wait
between pulses, and the stop rule gating the burst."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _workload():
    # 24 x 24 pixels (N = 576), M = 1100 atoms (9 blocks, ragged), K = 96
    return small_workload(nx=24, ny=24, n_freq=96, n_pulses=8,
                          dictionary="gaussian", n_atoms=1100, sparsity=0.03,
                          seed=21, dict_seed=4)


def _run(w, prec, problem, overlap, synth_ctas=0, device_data=False,
         steps=12, tol=0.0, simulate_between=False):
    import torch
    cfg = gpu_config(w, prec)
    cfg.overlap_synthesis = 1 if overlap else 0
    cfg.synth_ctas = int(synth_ctas)
    g = osar.Osar(cfg)
    track, _, c_true, data = problem
    if device_data:
        d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        torch.cuda.synchronize()
    sims = []
    for s in range(track.shape[0]):
        if device_data:
            g.push_pulse_dev(track[s], d.data_ptr() + s * w.n_freq * 16)
        else:
            g.push_pulse(track[s], data[s])
        g.iterate(steps, tol, want_count=False)
        if simulate_between:
            sims.append(g.simulate_pulse(track[(s + 3) % len(track)], c_true))
    g.synchronize()
    return g, sims


def _same(a, b):
    assert np.array_equal(a.coeffs(), b.coeffs())
    assert np.array_equal(a.gram(), b.gram())
    assert a.state() == b.state()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fp64"])
@pytest.mark.parametrize("synth_ctas", [0, 3])
def test_overlap_is_bitwise_neutral(prec, synth_ctas):
    w = _workload()
    problem = build_problem(w)
    ref, _ = _run(w, prec, problem, overlap=False)
    got, _ = _run(w, prec, problem, overlap=True, synth_ctas=synth_ctas)
    _same(ref, got)


def test_overlap_with_device_pulses_and_stop_rule():
    w = _workload()
    problem = build_problem(w)
    ref, _ = _run(w, "split_bf16", problem, overlap=False, steps=60, tol=1e-4)
    got, _ = _run(w, "split_bf16", problem, overlap=True, device_data=True,
                  steps=60, tol=1e-4)
    _same(ref, got)


def test_overlap_with_simulation_between_pushes():
    w = _workload()
    problem = build_problem(w)
    ref, s_ref = _run(w, "split_bf16", problem, overlap=False, simulate_between=True)
    got, s_got = _run(w, "split_bf16", problem, overlap=True, simulate_between=True)
    _same(ref, got)
    for a, b in zip(s_ref, s_got):
        assert np.array_equal(a, b)


def test_async_coefficient_reads_in_a_pipelined_loop():
    """Each pulse's image, read with coeffs_async while the next pulse is
    already queued, equals the image a synchronous loop reads."""
    import torch
    w = _workload()
    problem = build_problem(w)
    track, _, _, data = problem
    ref = osar.Osar(gpu_config(w, "split_bf16"))
    want = []
    for s in range(len(track)):
        ref.push_pulse(track[s], data[s])
        ref.iterate(12, 1e-4)
        want.append(ref.coeffs())
    g = osar.Osar(gpu_config(w, "split_bf16"))
    bufs = [torch.empty(w.m_atoms, dtype=torch.complex128).pin_memory()
            for _ in range(osar.COPY_SLOTS)]
    got = [None] * len(track)
    for s in range(len(track)):
        g.push_pulse(track[s], data[s])
        g.iterate(12, 1e-4, want_count=False)
        g.coeffs_async(bufs[s % osar.COPY_SLOTS].numpy(), slot=s % osar.COPY_SLOTS)
        if s >= 1:
            g.wait_coeffs((s - 1) % osar.COPY_SLOTS)
            got[s - 1] = bufs[(s - 1) % osar.COPY_SLOTS].numpy().copy()
    g.wait_coeffs((len(track) - 1) % osar.COPY_SLOTS)
    got[-1] = bufs[(len(track) - 1) % osar.COPY_SLOTS].numpy().copy()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    with pytest.raises(osar.OsarError):
        g.wait_coeffs(osar.COPY_SLOTS)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fp64"])
def test_overlap_alternating_main_and_side_synthesis(prec):
    # A host wait leaves the main stream idle, so the next push synthesises
    # in order on the main stream; the push after it goes to the side stream
    # again and must not start its phases while that synthesis still reads
    # the phase buffers.
    w = _workload()
    problem = build_problem(w)
    ref, _ = _run(w, prec, problem, overlap=False)
    cfg = gpu_config(w, prec)
    cfg.overlap_synthesis = 1
    g = osar.Osar(cfg)
    track, _, _, data = problem
    for s in range(track.shape[0]):
        g.push_pulse(track[s], data[s])
        g.iterate(12, 0.0, want_count=False)
        if s % 3 == 1:
            g.synchronize()
    g.synchronize()
    _same(ref, g)
