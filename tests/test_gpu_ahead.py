"""The Gram update run ahead (gram_ahead): each push forms A_n and
G_n = G_{n-1} + A_n^H A_n (Eqs. 12-13) on the side stream into a second
Gram buffer, beside the previous pulse's burst, and the main stream waits
for it and swaps buffers.  Only the schedule changes, so every result must
be bitwise the in-order run's, which the parity tests hold to the oracle:

* pulses queued without synchronisation (the update really runs beside the
  previous burst), every push ahead: coefficients, state, b and the whole
  Gram bitwise;
* schedules mixed push by push (ahead, in order, the model's choice),
  compared at every synchronisation;
* the pixel basis (no dictionary product: the side stream forms the phase
  planes and the update);
* checkpoints, non-white pulses, the setter's and the config's refusals."""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu


def _problem():
    # 2048 atoms: 136 packed Gram blocks over several CTA pairs
    w = small_workload(nx=32, ny=32, n_freq=128, n_pulses=8, span_deg=20.0,
                       dictionary="gaussian", n_atoms=2048, sparsity=0.02,
                       seed=21, dict_seed=7)
    track, _, _, data = build_problem(w)
    return w, track, data


def _ctx(w, ahead):
    cfg = gpu_config(w, "split_bf16")
    cfg.gram_ahead = ahead
    return osar.Osar(cfg)


def _same(a, b, tag):
    assert np.array_equal(a.coeffs(), b.coeffs()), tag
    assert a.state() == b.state(), tag
    assert np.array_equal(a.b(), b.b()), tag


def test_queued_pulses_ahead_are_bitwise_in_order():
    w, track, data = _problem()
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    for g in (ref, ahd):
        for s in range(track.shape[0]):
            g.push_pulse(track[s], data[s])
            g.iterate(20, want_count=False)
    _same(ref, ahd, "end")
    assert np.array_equal(ref.gram(), ahd.gram())
    assert ahd.profile_ahead() == track.shape[0]
    assert ref.profile_ahead() == 0


def test_mixed_schedules_are_bitwise_in_order():
    w, track, data = _problem()
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    modes = [2, 2, 0, 2, 1, 0, 0, 2]
    for s in range(track.shape[0]):
        ahd.set_gram_ahead(modes[s])
        before = ahd.profile_ahead()
        for g in (ref, ahd):
            g.push_pulse(track[s], data[s])
            g.iterate(12 if s % 2 else 20, 1e-6, want_count=False)
        if modes[s] == 2:
            assert ahd.profile_ahead() == before + 1, s
        if modes[s] == 0:
            assert ahd.profile_ahead() == before, s
        if s % 3 == 2:
            _same(ref, ahd, s)
    _same(ref, ahd, "end")
    assert np.array_equal(ref.gram(), ahd.gram())
    assert ahd.profile_ahead() >= 4


def test_refusals():
    w, _, _ = _problem()
    g = _ctx(w, 0)
    with pytest.raises(osar.OsarError) as e:
        g.set_gram_ahead(1)
    assert e.value.status == osar.OSAR_E_STATE
    h = _ctx(w, 1)
    with pytest.raises(osar.OsarError) as e:
        h.set_gram_ahead(3)
    assert e.value.status == osar.OSAR_E_INVALID
    h.set_gram_ahead(0)
    for prec, extra in [("fp32", {}), ("split_bf16", {"defer_gram": 1}),
                        ("split_bf16", {"overlap_synthesis": 0}),
                        ("split_bf16", {"pixel_gram": 1})]:
        cfg = gpu_config(w, prec)
        cfg.gram_ahead = 1
        for k, v in extra.items():
            setattr(cfg, k, v)
        with pytest.raises(osar.OsarError) as e:
            osar.Osar(cfg)
        assert e.value.status == osar.OSAR_E_INVALID, (prec, extra)



def test_checkpoint_resume_with_the_update_ahead(tmp_path):
    """A checkpoint taken between queued ahead pushes resumes bit for bit
    (the save waits for the Gram the next burst reads, in whichever
    buffer it sits)."""
    w, track, data = _problem()
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    half = track.shape[0] // 2
    for s in range(half):
        for g in (ref, ahd):
            g.push_pulse(track[s], data[s])
            g.iterate(20, want_count=False)
    path = str(tmp_path / "ahead.ckpt")
    ahd.save(path)
    ahd.close()
    cfg = gpu_config(w, "split_bf16")
    cfg.gram_ahead = 2
    res = osar.Osar.load(path, cfg)
    for s in range(half, track.shape[0]):
        for g in (ref, res):
            g.push_pulse(track[s], data[s])
            g.iterate(20, want_count=False)
    _same(ref, res, "resumed")
    assert np.array_equal(ref.gram(), res.gram())


def test_non_white_pulses_ahead_are_bitwise_in_order():
    """Pulses with their own noise variances (the phase rows weighted by
    1 / sigma_k on the stream that forms them) keep the in-order results."""
    w, track, data = _problem()
    var = np.random.default_rng(3).uniform(0.5, 2.0, size=(track.shape[0], w.n_freq))
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    for g in (ref, ahd):
        for s in range(track.shape[0]):
            g.push_pulse(track[s], data[s], noise_var=var[s] if s % 2 else None)
            g.iterate(20, want_count=False)
    _same(ref, ahd, "end")
    assert np.array_equal(ref.gram(), ahd.gram())


def test_pixel_basis_ahead_is_bitwise_in_order():
    w = small_workload(nx=48, ny=48, n_freq=96, n_pulses=6, span_deg=20.0,
                       sparsity=0.03, seed=23)
    track, _, _, data = build_problem(w)
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    for g in (ref, ahd):
        for s in range(track.shape[0]):
            g.push_pulse(track[s], data[s])
            g.iterate(15, want_count=False)
    _same(ref, ahd, "end")
    assert np.array_equal(ref.gram(), ahd.gram())
    assert ahd.profile_ahead() == track.shape[0]


def test_adjoint_after_ahead_pushes_is_bitwise_in_order():
    """osar_unroll_grad replays a cached CUDA graph of its passes; after the
    Gram buffers swap it must read the new Gram (the passes take its
    address from device memory)."""
    w, track, data = _problem()
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    c_true = np.zeros(w.m_atoms, complex)
    c_true[::97] = 1.0
    out = {}
    for tag, g in (("ref", ref), ("ahd", ahd)):
        res = []
        for s in range(4):
            g.push_pulse(track[s], data[s])
            g.iterate(10, want_count=False)
            st = g.state()
            res.append(g.unroll_grad(8, 4, st["lambda"], 1.0 / st["lipschitz"],
                                     g.coeffs(), c_true))
        out[tag] = res
    for a, b in zip(out["ref"], out["ahd"]):
        assert a["loss"] == b["loss"]
        assert a["d_lambda"] == b["d_lambda"] and a["d_tau"] == b["d_tau"]
        assert np.array_equal(a["d_b"], b["d_b"])


def test_captured_burst_follows_the_swaps():
    """A burst captured once in a CUDA graph and replayed for later pulses
    reads each pulse's Gram, in whichever buffer it sits."""
    torch = pytest.importorskip("torch")
    w, track, data = _problem()
    stream = torch.cuda.Stream()

    def ctx(ahead):
        cfg = gpu_config(w, "split_bf16")
        cfg.gram_ahead = ahead
        cfg.cuda_stream = stream.cuda_stream
        return osar.Osar(cfg)

    eager, replay = ctx(0), ctx(2)
    graph = None
    for s in range(track.shape[0]):
        for g in (eager, replay):
            g.push_pulse(track[s], data[s])
            g.iterate(4, want_count=False)
        eager.iterate(6, want_count=False)
        if graph is None:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                replay.iterate(6, want_count=False)
        with torch.cuda.stream(stream):
            graph.replay()
        stream.synchronize()
        assert np.array_equal(eager.coeffs(), replay.coeffs()), s
        assert eager.state() == replay.state(), s
    assert replay.profile_ahead() == track.shape[0]


def test_edgelet_dictionary_ahead_is_bitwise_in_order():
    """Edgelet blocks (sums of phase rows, no GEMM) formed on the side
    stream with the update run ahead."""
    w = small_workload(nx=24, ny=24, n_freq=64, n_pulses=6, span_deg=20.0,
                       dictionary="edgelet", edgelet_lengths=(4,),
                       edgelet_angles=(0.0, 90.0), sparsity=0.02, seed=25)
    track, _, _, data = build_problem(w)
    ref, ahd = _ctx(w, 0), _ctx(w, 2)
    for g in (ref, ahd):
        for s in range(track.shape[0]):
            g.push_pulse(track[s], data[s])
            g.iterate(15, want_count=False)
    _same(ref, ahd, "end")
    assert np.array_equal(ref.gram(), ahd.gram())
    assert ahd.profile_ahead() == track.shape[0]


@pytest.mark.parametrize("tc_pairs,power_gram", [(0, 0), (1, 1), (2, 0)])
def test_other_kernel_choices_ahead_are_bitwise_in_order(tc_pairs, power_gram):
    """The update run ahead on single-SM tiles or SM pairs, with or without
    the power step in its epilogue."""
    w, track, data = _problem()
    ctxs = []
    for ahead in (0, 2):
        cfg = gpu_config(w, "split_bf16")
        cfg.gram_ahead = ahead
        cfg.tc_pairs = tc_pairs
        cfg.fuse_power_gram = power_gram
        ctxs.append(osar.Osar(cfg))
    ref, ahd = ctxs
    for g in (ref, ahd):
        for s in range(4):
            g.push_pulse(track[s], data[s])
            g.iterate(12, want_count=False)
    _same(ref, ahd, (tc_pairs, power_gram))
    assert np.array_equal(ref.gram(), ahd.gram())


def test_static_gram_apply_reads_the_current_buffer():
    """The allocation-free Gram apply after ahead pushes (the Gram then sits
    in either buffer) equals the allocating apply bit for bit."""
    torch = pytest.importorskip("torch")
    w, track, data = _problem()
    g = _ctx(w, 2)
    rng = np.random.default_rng(8)
    for s in range(3):
        g.push_pulse(track[s], data[s])
        g.iterate(5, want_count=False)
        x = rng.standard_normal(w.m_atoms) + 1j * rng.standard_normal(w.m_atoms)
        ref = g.gram_apply(x)
        xd = torch.from_numpy(x).to("cuda")
        yd = torch.empty_like(xd)
        torch.cuda.synchronize()
        g.gram_apply_static(xd.data_ptr(), yd.data_ptr())
        g.synchronize()
        assert np.array_equal(yd.cpu().numpy(), ref), s
    assert g.profile_ahead() == 3


def test_lambda_path_ahead_is_bitwise_in_order():
    """Several solutions sharing one Gram (the lambda path) with the update
    run ahead."""
    w, track, data = _problem()
    lams = np.asarray([0.02, 0.05, 0.11], dtype=np.float64)
    ctxs = []
    for ahead in (0, 2):
        cfg = gpu_config(w, "split_bf16")
        cfg.n_lambdas = len(lams)
        cfg.lambda_list = lams.ctypes.data
        cfg.gram_ahead = ahead
        ctxs.append(osar.Osar(cfg))
    ref, ahd = ctxs
    for g in (ref, ahd):
        for s in range(5):
            g.push_pulse(track[s], data[s])
            g.iterate(12, want_count=False)
    for l in range(len(lams)):
        a, b = ref.lambda_state(l), ahd.lambda_state(l)
        assert np.array_equal(a["coeffs"], b["coeffs"]), l
        assert a["lambda"] == b["lambda"] and a["t"] == b["t"], l
    assert np.array_equal(ref.gram(), ahd.gram())
    assert ahd.profile_ahead() == 5
