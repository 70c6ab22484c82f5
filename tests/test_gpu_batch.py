"""Batching form: uneven scenes in one osar_batch against their own FP64
oracles (and against separate single-scene contexts), with per-scene active
masks, graph-replayed bursts, the tol stop rule and the matvec autotuner.
Tolerances as in test_gpu_parity."""
import os

import numpy as np
import pytest

from oracle import osar_oracle as orc
from paper_2603_08582_gb300 import osar, synth
from tests.helpers import (small_workload, build_problem, oracle_config, rel_err,
                           assert_close, assert_coeffs, SUPPORT_DELTA)
from tests.gpu_helpers import gpu_config

pytestmark = pytest.mark.gpu

TOL_C = {"fp64": 1e-7, "fp32": 1e-4, "split_bf16": 1e-3}


def _scenes(seed=0):
    rng = np.random.default_rng(seed)
    shapes = [(8, 8, 16), (12, 12, 24), (16, 16, 20), (9, 13, 28), (20, 20, 32)]
    ws = []
    for i, (nx, ny, k) in enumerate(shapes):
        ws.append(small_workload(
            nx=nx, ny=ny, n_freq=k, n_pulses=int(rng.integers(4, 8)),
            span_deg=float(rng.uniform(15, 35)), radius=float(rng.uniform(800, 1200)),
            sparsity=float(rng.uniform(0.03, 0.08)), seed=100 + i))
    return ws


def _run(prec, steps=8, tol=0.0, ws=None, check_every=True):
    ws = ws or _scenes()
    probs = [build_problem(w) for w in ws]
    oracles = [orc.OnlineFista(oracle_config(w, None)) for w in ws]
    batch = osar.OsarBatch([gpu_config(w, prec) for w in ws])
    P = max(w.n_pulses for w in ws)
    for s in range(P):
        active = [1 if s < w.n_pulses else 0 for w in ws]
        gam = np.zeros((len(ws), 3))
        data = []
        for q, (w, pr) in enumerate(zip(ws, probs)):
            if active[q]:
                gam[q] = pr[0][s]
                data.append(pr[3][s])
                oracles[q].push_pulse(pr[0][s], pr[3][s])
            else:
                data.append(None)
        batch.push(active, gam, data)
        counts = batch.iterate(steps, tol)
        for q, w in enumerate(ws):
            if active[q]:
                n_o = oracles[q].iterate(steps, tol)
                assert counts[q] == n_o, (q, counts[q], n_o)
            if check_every or s == P - 1:
                assert_coeffs(batch.coeffs(q), oracles[q].s, TOL_C[prec],
                              SUPPORT_DELTA[prec], f"c {prec} pulse {s} scene {q}")
    return ws, oracles, batch


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_batch_matches_per_scene_oracles(prec):
    ws, oracles, batch = _run(prec)
    for q, w in enumerate(ws):
        st = batch.state(q)
        assert st["n"] == oracles[q].s.n
        assert abs(st["lipschitz"] - oracles[q].s.lip) <= 1e-4 * oracles[q].s.lip
        assert abs(st["t"] - oracles[q].s.t) <= 1e-9 * oracles[q].s.t


def test_batch_tolerance_stop_per_scene():
    _run("fp64", steps=200, tol=1e-5, check_every=False)


def test_batch_equals_single_contexts_and_graph_replay():
    ws = _scenes(seed=3)
    probs = [build_problem(w) for w in ws]
    batch = osar.OsarBatch([gpu_config(w, "fp64") for w in ws])
    singles = [osar.Osar(gpu_config(w, "fp64")) for w in ws]
    for s in range(3):
        gam = np.stack([pr[0][s] for pr in probs])
        data = [pr[3][s] for pr in probs]
        batch.push([1] * len(ws), gam, data)
        batch.iterate(3)            # graph captured for 3 steps
        batch.iterate(3)            # replayed
        for q, g in enumerate(singles):
            g.push_pulse(probs[q][0][s], probs[q][3][s])
            g.iterate(6)
            # same kernels; the batch's matvec segments group the partial
            # sums differently, so FP64 rounding differs at ~1e-11
            assert rel_err(batch.coeffs(q), g.coeffs()) <= 1e-9


def test_batch_autotune_keeps_results(tmp_path):
    os.environ["OSAR_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        ws = _scenes(seed=5)
        probs = [build_problem(w) for w in ws]
        a = osar.OsarBatch([gpu_config(w, "fp64") for w in ws])
        b = osar.OsarBatch([gpu_config(w, "fp64") for w in ws])
        chosen = b.autotune()
        assert chosen in (1, 2, 4, 8, 16)
        assert b.info()["segment_blocks"] == chosen
        for s in range(3):
            gam = np.stack([pr[0][s] for pr in probs])
            data = [pr[3][s] for pr in probs]
            for x in (a, b):
                x.push([1] * len(ws), gam, data)
                x.iterate(5)
        for q in range(len(ws)):
            assert rel_err(a.coeffs(q), b.coeffs(q)) <= 1e-12
        c = osar.OsarBatch([gpu_config(w, "fp64") for w in ws])
        assert c.info()["segment_blocks"] == chosen       # read from the cache
    finally:
        del os.environ["OSAR_TUNE_CACHE"]


def test_batch_autotune_gram_order(tmp_path):
    """The Gram update's tile order is timed before the first pulse (the
    timed updates add exact zeros: the results equal an untuned batch's) and
    kept after it; the choice is cached with the segment size."""
    os.environ["OSAR_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        ws = _scenes(seed=6)
        probs = [build_problem(w) for w in ws]
        a = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
        b = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
        b.autotune()
        t = b.tuning()
        assert t["gram_superblock"] in (4, 8, 16, 32)
        assert 0.0 < t["gram_ms_chosen"] <= t["gram_ms_default"]
        for s in range(3):
            gam = np.stack([pr[0][s] for pr in probs])
            data = [pr[3][s] for pr in probs]
            for x in (a, b):
                x.push([1] * len(ws), gam, data)
                x.iterate(6)
        for q in range(len(ws)):
            # the segment size regroups the matvec's FP32 partial sums
            assert rel_err(b.coeffs(q), a.coeffs(q)) <= 1e-6
        c = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
        tc = c.tuning()                                  # read from the cache
        assert (tc["segment_blocks"], tc["gram_superblock"], tc["gram_largest_first"]) == \
            (t["segment_blocks"], t["gram_superblock"], t["gram_largest_first"])
        # after a pulse the order is kept and the Gram update is not timed
        del os.environ["OSAR_TUNE_CACHE"]
        d = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
        gam = np.stack([pr[0][0] for pr in probs])
        d.push([1] * len(ws), gam, [pr[3][0] for pr in probs])
        d.autotune()
        td = d.tuning()
        assert td["gram_ms_chosen"] == 0.0 and td["gram_superblock"] == 8
        d.iterate(6)
        e = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
        e.push([1] * len(ws), gam, [pr[3][0] for pr in probs])
        e.iterate(6)
        for q in range(len(ws)):
            assert rel_err(d.coeffs(q), e.coeffs(q)) <= 1e-6
    finally:
        os.environ.pop("OSAR_TUNE_CACHE", None)


def test_batch_96_uneven_scenes_split_bf16():
    """The batching workload: 96 scenes, sides 32..96, K = 256, own tracks;
    three pulses each in split-BF16, checked against the FP64 oracle on four
    scenes of different sizes."""
    ws = synth.batch_workloads(96)
    track = [synth.workload_track(w) for w in ws]
    rng = np.random.default_rng(1)
    batch = osar.OsarBatch([gpu_config(w, "split_bf16") for w in ws])
    chosen = batch.autotune()
    assert chosen in (1, 2, 4, 8, 16)
    sides = sorted({w.nx for w in ws})
    pick = [next(q for q, w in enumerate(ws) if w.nx == sd) for sd in sides[:4]]
    oracles = {q: orc.OnlineFista(oracle_config(ws[q], None)) for q in pick}
    probs = {q: build_problem(ws[q]) for q in pick}
    for s in range(3):
        gam = np.stack([t[s] for t in track])
        data = []
        for q, w in enumerate(ws):
            if q in probs:
                data.append(probs[q][3][s])
            else:
                data.append(rng.standard_normal(w.n_freq) + 1j * rng.standard_normal(w.n_freq))
        batch.push([1] * len(ws), gam, data)
        batch.iterate(10)
        for q in pick:
            oracles[q].push_pulse(probs[q][0][s], probs[q][3][s])
            oracles[q].iterate(10)
    for q in pick:
        assert_coeffs(batch.coeffs(q), oracles[q].s, 1e-3,
                      SUPPORT_DELTA["split_bf16"], f"c scene {q} side {ws[q].nx}")
