"""The allocation-free Gram apply, osar_gram_apply_static.

Callers that must not allocate device memory once they are running (fixed
memory budgets on embedded or flight systems, hosts that hand out every
buffer from their own pool) use this entry point: they pass x and y in
device memory and the matvec's scratch comes from a static array inside the
library.  These tests check it against the allocating entry point,
osar_gram_apply, which runs the same kernels on the same data, so the two
must agree bit for bit: on two calls in a row (the shared array keeps the
previous call's contents), after a larger context has filled more of the
array than a smaller one uses, at the size limit itself, in every precision
and in the pixel-space Gram form.  They also check that a call allocates no
device memory, and the clear rejections: a Gram beyond the array, and
vectors that are not device memory of this GPU or not 16-byte aligned.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2603_08582_gb300 import osar
from tests.helpers import small_workload, build_problem
from tests.gpu_helpers import gpu_config

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _context(prec, nx=32, ny=32, n_freq=48, pulses=4, **kw):
    w = small_workload(nx=nx, ny=ny, n_freq=n_freq, n_pulses=pulses, seed=17, **kw)
    track, dic, c_true, data = build_problem(w)
    cfg = gpu_config(w, prec)
    if kw.get("dictionary") == "edgelet":
        cfg.pixel_gram = 1
    g = osar.Osar(cfg)
    for s in range(w.n_pulses):
        g.push_pulse(track[s], data[s])
        g.iterate(3)
    return g


def _dim(g):
    # the apply works on the Gram the context stores: G_n (M atoms), or P_n
    # (N pixels) in the pixel-space form
    return g.gram_dim


def _static(g, x):
    x_dev = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    y_dev = torch.full(x_dev.shape, complex(np.nan, np.nan),
                       dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
    g.synchronize()
    return y_dev.cpu().numpy()


def _vec(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_bf16"])
def test_static_apply_equals_allocating_apply_twice(prec):
    g = _context(prec)
    rng = np.random.default_rng(5)
    for _ in range(2):
        x = _vec(rng, _dim(g))
        y = _static(g, x)
        assert np.array_equal(y, g.gram_apply(x))


def test_static_apply_after_a_larger_context_and_at_the_limit():
    """A 64 x 64 pixel-basis context (M = 4096, the stated limit) in FP64
    fills the most scratch; a smaller ragged context's apply that follows
    must not read any of it."""
    rng = np.random.default_rng(9)
    big = _context("fp64", nx=64, ny=64, n_freq=24, pulses=2)
    assert _dim(big) == 4096
    xb = _vec(rng, 4096)
    assert np.array_equal(_static(big, xb), big.gram_apply(xb))
    small = _context("fp64", nx=13, ny=11, n_freq=20, pulses=3)
    for _ in range(2):
        xs = _vec(rng, _dim(small))
        assert np.array_equal(_static(small, xs), small.gram_apply(xs))
    # and the large one again after the small one
    assert np.array_equal(_static(big, xb), big.gram_apply(xb))


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_static_apply_pixel_space_form(prec):
    g = _context(prec, nx=16, ny=12, n_freq=32, dictionary="edgelet",
                 edgelet_lengths=(4,), edgelet_angles=(0.0, 90.0))
    assert _dim(g) == 16 * 12
    rng = np.random.default_rng(2)
    for _ in range(2):
        x = _vec(rng, _dim(g))
        assert np.array_equal(_static(g, x), g.gram_apply(x))


def test_static_apply_allocates_no_device_memory():
    g = _context("split_bf16")
    rng = np.random.default_rng(4)
    n = _dim(g)
    x_dev = torch.from_numpy(_vec(rng, n)).to("cuda")
    y_dev = torch.empty_like(x_dev)
    g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
    g.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
    g.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_apply_rejects_gram_beyond_static_scratch():
    w = small_workload(nx=128, ny=64, n_freq=16, n_pulses=1)
    g = osar.Osar(gpu_config(w, "fp32"))
    x_dev = torch.zeros(w.m_atoms, dtype=torch.complex128, device="cuda")
    y_dev = torch.zeros_like(x_dev)
    with pytest.raises(osar.OsarError) as ei:
        g.gram_apply_static(x_dev.data_ptr(), y_dev.data_ptr())
    assert ei.value.status == osar.OSAR_E_INVALID
    assert "static" in str(ei.value)


def test_static_apply_rejects_host_and_unaligned_vectors():
    g = _context("fp32", nx=16, ny=16, n_freq=24, pulses=2)
    n = _dim(g)
    x_dev = torch.zeros(n + 1, dtype=torch.complex128, device="cuda")
    y_dev = torch.zeros_like(x_dev)
    host = np.zeros(n, dtype=np.complex128)
    pinned = torch.zeros(n, dtype=torch.complex128).pin_memory()
    cases = [
        (host.ctypes.data, y_dev.data_ptr(), "host"),
        (x_dev.data_ptr(), host.ctypes.data, "host"),
        (pinned.data_ptr(), y_dev.data_ptr(), "page-locked"),
        (x_dev.data_ptr() + 8, y_dev.data_ptr(), "aligned"),
        (x_dev.data_ptr(), y_dev.data_ptr() + 8, "aligned"),
    ]
    for xp, yp, word in cases:
        with pytest.raises(osar.OsarError) as ei:
            g.gram_apply_static(xp, yp)
        assert ei.value.status == osar.OSAR_E_INVALID
        assert word in str(ei.value)
    # nothing was launched: the context still works
    x = _vec(np.random.default_rng(1), n)
    assert np.array_equal(_static(g, x), g.gram_apply(x))
