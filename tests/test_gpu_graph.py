"""Bursts replayed from a CUDA graph: osar_iterate only queues kernels on the
context's stream (no allocation, no synchronisation when no count is
asked for), so a caller can capture a burst once and replay it for every
later pulse.  The replayed run must be bitwise the eager one, for the
stored Gram (split-BF16, FP64) and the pixel-space Gram form, with the stop
rule deciding on the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _workload(kind):
    if kind == "pixel_gram":
        return small_workload(nx=12, ny=12, n_freq=40, n_pulses=6,
                              dictionary="edgelet", edgelet_lengths=(4,),
                              edgelet_angles=(0.0, 90.0), sparsity=0.02, seed=9)
    return small_workload(nx=16, ny=16, n_freq=48, n_pulses=6,
                          dictionary="gaussian", n_atoms=600, sparsity=0.03,
                          seed=14, dict_seed=5)


@pytest.mark.parametrize("kind,prec", [("stored", "split_bf16"), ("stored", "fp64"),
                                       ("pixel_gram", "split_bf16")])
def test_replayed_bursts_are_the_eager_ones(kind, prec):
    w = _workload(kind)
    track, _, _, data = build_problem(w)
    stream = torch.cuda.Stream()

    def ctx():
        cfg = gpu_config(w, prec)
        cfg.cuda_stream = stream.cuda_stream
        cfg.pixel_gram = 1 if kind == "pixel_gram" else 0
        return osar.Osar(cfg)

    eager, replay = ctx(), ctx()
    graph = None
    for s in range(track.shape[0]):
        for g in (eager, replay):
            g.push_pulse(track[s], data[s])
            g.iterate(4, 1e-5, want_count=False)   # starts the burst
        eager.iterate(6, 1e-5, want_count=False)
        if graph is None:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                replay.iterate(6, 1e-5, want_count=False)
        with torch.cuda.stream(stream):   # replay in order on the context's stream
            graph.replay()
        stream.synchronize()
        assert np.array_equal(eager.coeffs(), replay.coeffs()), s
        assert eager.state() == replay.state(), s
