"""CPU-side checks of the C ABI: libosar.so builds for sm_103a, loads, exports
every function include/osar.h declares, and its host-only logic (defaults,
argument validation) behaves as documented.  No kernel runs here."""
import ctypes as C
import os
import re

import pytest

from paper_2603_08582_gb300 import build, osar

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "osar.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return osar.load_library()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(osar_[a-z_]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(osar.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_config_defaults_and_layout(lib):
    cfg = osar.default_config()
    assert (cfg.nx, cfg.ny, cfg.n_freq) == (32, 32, 128)
    assert cfg.pixel_m == 1.0
    assert cfg.f_lo_hz == 9.9e9 and cfg.f_hi_hz == 10.1e9
    assert cfg.precision == osar.OSAR_FP64
    assert cfg.dict_kind == osar.OSAR_DICT_IDENTITY
    assert cfg.lam == 0.05 and cfg.lambda_relative == 1
    assert (cfg.power_iters_first, cfg.power_iters) == (30, 4)
    assert cfg.lipschitz_margin == 0.01
    assert cfg.restart_momentum == 0 and cfg.compensated == 1
    assert cfg.cuda_stream is None
    assert cfg.overlap_synthesis == 1 and cfg.synth_ctas == 0
    assert cfg.tc_pairs == 3 and cfg.fuse_first_step == 1
    assert cfg.n_lambdas == 1 and cfg.lambda_list is None
    assert cfg.defer_gram == 0 and cfg.guard_bytes == 0
    assert cfg.fuse_power_gram == 1 and cfg.pixel_gram == 0
    assert cfg.gram_superblock == 0 and cfg.gram_ahead == 0


def test_config_struct_layout_matches_the_header(tmp_path):
    """The binding's osar_config and osar_metrics have the C structs' size
    and field offsets (a C program compiled against include/osar.h prints
    them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"osar_config": osar.OsarConfig, "osar_metrics": osar.OsarMetrics}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "osar.h"',
             "int main(void) {"]
    for cname, ct in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in ct._fields_:
            cf = "lambda" if f == "lam" else f
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        cname, what, value = line.split()
        ct = structs[cname]
        want = C.sizeof(ct) if what == "size" else getattr(ct, what).offset
        assert int(value) == want, line


@pytest.mark.parametrize("changes", [
    {"defer_gram": 2},
    {"defer_gram": 1},                                   # FP64, identity dictionary
    {"defer_gram": 1, "precision": osar.OSAR_SPLIT_BF16},  # no dictionary
    {"defer_gram": 1, "precision": osar.OSAR_FP32,
     "dict_kind": osar.OSAR_DICT_GAUSSIAN, "n_atoms": 300},
    {"defer_gram": 1, "precision": osar.OSAR_SPLIT_BF16,
     "dict_kind": osar.OSAR_DICT_GAUSSIAN, "n_atoms": 300, "overlap_synthesis": 0},
])
def test_create_rejects_unsupported_deferred_update(lib, changes):
    cfg = osar.default_config()
    for k, v in changes.items():
        setattr(cfg, k, v)
    h = C.c_void_p()
    assert lib.osar_create(C.byref(cfg), C.byref(h)) == osar.OSAR_E_INVALID
    assert h.value is None
    assert b"defer_gram" in lib.osar_last_error(None)


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("n_freq", 0), ("pixel_m", -1.0), ("f_lo_hz", 0.0),
    ("precision", 7), ("dict_kind", 9), ("power_iters_first", 0),
    ("lam", float("nan")), ("lipschitz_margin", -0.5),
    ("overlap_synthesis", 2), ("synth_ctas", -1), ("tc_pairs", 4),
    ("fuse_first_step", 2), ("fuse_power_gram", 2), ("pixel_gram", 2),
    ("pixel_gram", 1),  # the pixel-space Gram form needs a dictionary
    ("gram_superblock", -1), ("gram_superblock", 65),
    ("gram_ahead", -1), ("gram_ahead", 3),
    ("gram_ahead", 1),  # the default config is FP64 with no dictionary
    ("n_lambdas", 0),
    ("n_lambdas", 9),
    ("n_lambdas", 2),  # > 1 without a lambda_list
    ("guard_bytes", -256), ("guard_bytes", 100), ("guard_bytes", 2 << 20),
])
def test_create_rejects_invalid_config_before_any_device_work(lib, field, value):
    cfg = osar.default_config()
    setattr(cfg, field, value)
    h = C.c_void_p()
    st = lib.osar_create(C.byref(cfg), C.byref(h))
    assert st == osar.OSAR_E_INVALID
    assert h.value is None
    assert len(lib.osar_last_error(None)) > 0


@pytest.mark.parametrize("lengths,angles,n_atoms", [
    ([], [0.0], 0), ([4], [], 0), ([0], [0.0], 0), ([65], [0.0], 0),
    ([4], [30.0], 0), ([4], [360.0], 0), ([4], [-45.0], 0),
    ([4], [0.0, 90.0], 7),          # n_atoms must be 0 or 2 x pixels
])
def test_create_rejects_invalid_edgelets(lib, lengths, angles, n_atoms):
    cfg = osar.make_config(8, 8, 16, 9.9e9, 10.1e9, dictionary="edgelet",
                           edgelet_lengths=lengths or [1], edgelet_angles=angles or [0.0])
    if not lengths:
        cfg.n_edgelet_lengths = 0
    if not angles:
        cfg.n_edgelet_angles = 0
    cfg.n_atoms = n_atoms
    h = C.c_void_p()
    assert lib.osar_create(C.byref(cfg), C.byref(h)) == osar.OSAR_E_INVALID
    assert h.value is None


def test_create_rejects_missing_host_dictionary(lib):
    cfg = osar.default_config()
    cfg.dict_kind = osar.OSAR_DICT_HOST
    cfg.n_atoms = 10
    h = C.c_void_p()
    assert lib.osar_create(C.byref(cfg), C.byref(h)) == osar.OSAR_E_INVALID


def test_null_context_calls_are_rejected(lib):
    assert lib.osar_destroy(None) == osar.OSAR_OK
    assert lib.osar_iterate(None, 1, 0.0, None) == osar.OSAR_E_INVALID
    assert lib.osar_synchronize(None) == osar.OSAR_E_INVALID
    assert lib.osar_probe_bounded_wait(None, 10**8) == osar.OSAR_E_INVALID
    assert b"libosar" in lib.osar_version()


def test_sources_have_no_cpu_fallback():
    """The product package never reaches the oracle."""
    pkg = os.path.join(ROOT, "paper_2603_08582_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), f
