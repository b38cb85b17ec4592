"""Host-side checks of the C ABI: the library loads, exports every symbol that
include/cola.h declares, and validates arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int32_t|uint64_t|const char\*)\s+(cola_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol():
    import paper_1509_04685_gb300 as C
    names = _declared()
    assert len(names) >= 14
    lib = ctypes.CDLL(C.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size_and_validation():
    import paper_1509_04685_gb300 as C
    cfg = C.make_config(32, 96, 128.0, 0.05)
    assert C.cola_workspace_size(cfg) > 96**3 * 8
    for bad in (dict(nq=7), dict(ng=14), dict(ng=3), dict(ng=8192)):
        kw = dict(nq=32, ng=96)
        kw.update(bad)
        with pytest.raises(C.ColaError) as e:
            C.cola_workspace_size(C.make_config(kw["nq"], kw["ng"], 128.0, 0.05))
        assert e.value.code in (-1, -3)
    with pytest.raises(C.ColaError):
        C.cola_workspace_size(C.make_config(32, 96, -1.0, 0.05))
    with pytest.raises(C.ColaError):
        C.cola_workspace_size(C.make_config(32, 96, 128.0, 0.05, n_steps=1))


def test_entry_points_reject_bad_arguments_without_launching():
    import paper_1509_04685_gb300 as C
    L = C.LIB
    cfg = C.make_config(8, 24, 32.0, 0.05)
    size = C.cola_workspace_size(cfg)
    fake = 1 << 40  # never dereferenced: every call below fails validation first
    st = C.cola_state(fake, fake, fake, fake)
    assert L.cola_step(ctypes.byref(cfg), ctypes.byref(st), 40, fake, size, None) == -1
    assert L.cola_step(ctypes.byref(cfg), ctypes.byref(st), -1, fake, size, None) == -1
    assert L.cola_step(ctypes.byref(cfg), ctypes.byref(st), 0, fake, size - 1, None) == -2
    assert L.cola_step(ctypes.byref(cfg), ctypes.byref(st), 0, fake + 8, size, None) == -1
    assert L.cola_pm_force(ctypes.byref(cfg), ctypes.byref(st), 0.5, None, fake, size, None) == -1
    assert L.cola_power_spectrum(ctypes.byref(cfg), ctypes.byref(st), 0, 0.05, 48, 0, fake, fake, fake, 24,
                                 fake, size, None) == -3  # ng_pk > ng
    assert L.cola_power_spectrum(ctypes.byref(cfg), ctypes.byref(st), 0, 0.05, 24, 0, fake, fake, fake, 11,
                                 fake, size, None) == -1  # nbins != ng_pk/2
    hs = C.cola_state(fake, fake, fake, fake)
    assert L.cola_step_host(ctypes.byref(cfg), ctypes.byref(hs), ctypes.byref(st), 40, fake, size, None) == -1
    assert L.cola_step_host(ctypes.byref(cfg), ctypes.byref(hs), ctypes.byref(st), 0, fake, size - 1, None) == -2
    assert L.cola_step_host(ctypes.byref(cfg), None, ctypes.byref(st), 0, fake, size, None) == -1
    for flags in (4 | 1, 4 | 2, 8):
        assert L.cola_power_spectrum(ctypes.byref(cfg), ctypes.byref(st), 0, 0.05, 24, flags, fake, fake, fake, 12,
                                     fake, size, None) == -1
    assert L.cola_power_multipoles(ctypes.byref(cfg), ctypes.byref(st), 0, 0.05, 24, 4, fake, fake, fake, fake, fake,
                                   12, fake, size, None) == -1
    assert C.cola_launch_count() == 0
    assert C.cola_strerror(-6).startswith("non-finite")


def test_particle_set_traversal_validates_its_arguments():
    import paper_1509_04685_gb300 as C
    for edge, bk in ((-32, 8), (16, 8), (48, 8), (96, 16), (8192, 8), (64, 4), (64, 128), (64, 12), (512, 512)):
        assert C.LIB.cola_particle_set_traversal(edge, bk) == -1
    for edge, bk in ((32, 8), (128, 16), (4096, 32), (256, 256), (0, 0)):  # 0 restores the default
        assert C.LIB.cola_particle_set_traversal(edge, bk) == 0


def test_fof_entry_points_validate_before_launching():
    import paper_1509_04685_gb300 as C
    L = C.LIB
    cfg = C.make_config(16, 48, 64.0, 0.05)
    fsize = C.cola_fof_workspace_size(cfg)
    assert fsize > 16**3 * 24
    fake = 1 << 40
    st = C.cola_state(fake, fake, fake, fake)
    call = lambda b, g, ws, n: L.cola_fof(ctypes.byref(cfg), ctypes.byref(st), b, g, ws, n, None)
    assert call(0.5, fake, fake, fsize) == -1
    assert call(0.0, fake, fake, fsize) == -1
    assert call(0.2, None, fake, fsize) == -1
    assert call(0.2, fake, fake, fsize - 1) == -2
    assert L.cola_fof_halos(ctypes.byref(cfg), fake, 0, fake, fake, fake, fake, fsize, None) == -1
    assert L.cola_mass_function(ctypes.byref(cfg), fake, fake, 10, 12.0, 0.0, 5, fake, None) == -1
    assert C.cola_launch_count() == 0


def test_package_refuses_to_import_without_the_cuda_library(tmp_path):
    # no fallback: a copy of the package without its built library does not import
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_1509_04685_gb300")
    dst = tmp_path / "paper_1509_04685_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    r = subprocess.run([sys.executable, "-c", "import paper_1509_04685_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "COLA CUDA library not built" in r.stderr


def test_package_sources_do_not_reach_the_oracle():
    # the product path neither imports nor runs anything under oracle/
    src = os.path.join(ROOT, "paper_1509_04685_gb300")
    for dirpath, _, files in os.walk(src):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
                mods = "|".join(m[:-3] for m in os.listdir(os.path.join(ROOT, "oracle")) if m.endswith(".py"))
                assert not re.search(rf"\boracle\.({mods})\b", text), f
                assert "oracle/" not in text and "import_module(\"oracle" not in text, f


def test_binding_argument_counts_match_the_header():
    # every declared entry point is bound with as many arguments as the header gives it
    import paper_1509_04685_gb300 as C
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    decls = re.findall(r"^\s*(?:int|int32_t|uint64_t|const char\*|void)\s+(cola_\w+)\s*\(([^;]*?)\)\s*;", text, re.M)
    assert len(decls) >= 30
    checked = 0
    for name, params in decls:
        fn = getattr(C.LIB, name)
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        if fn.argtypes is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
            checked += 1
    assert checked >= 25


def test_checkpoint_size_and_header_checks_without_copying():
    # the buffer size and every header check run before any copy
    import numpy as np

    import paper_1509_04685_gb300 as C
    L = C.LIB
    cfg = C.make_config(8, 24, 32.0, 0.05)
    n = C.cola_checkpoint_bytes(cfg)
    assert n == 256 + 4 * 3 * 8**3 * 4
    fake = 1 << 40
    st = C.cola_state(fake, fake, fake, fake)
    buf = np.zeros(n, np.uint8)
    node = ctypes.c_int32(-1)
    p = buf.ctypes.data
    assert L.cola_checkpoint_load(ctypes.byref(cfg), p, n, ctypes.byref(st), ctypes.byref(node), None) == -1  # no magic
    assert L.cola_checkpoint_save(ctypes.byref(cfg), ctypes.byref(st), 40, p, n, None) == -1  # node out of range
    assert L.cola_checkpoint_save(ctypes.byref(cfg), ctypes.byref(st), 3, p, n - 1, None) == -1  # short buffer
    assert L.cola_checkpoint_load(ctypes.byref(cfg), p, n - 1, ctypes.byref(st), ctypes.byref(node), None) == -1
    assert node.value == -1


def test_checks_entry_points_without_launching():
    # the product build carries no device bounds checks; the probe hook refuses
    # anything outside its 64-int area before launching
    import paper_1509_04685_gb300 as C
    assert C.LIB.cola_checks_enabled() == 0
    for index, n in ((-1, 8), (64, 64), (3, 0), (3, 65), (8, 8)):
        assert C.LIB.cola_checks_probe(index, n, 1 << 20, 1 << 20, None) == -1
    assert C.LIB.cola_checks_probe(0, 8, None, 1 << 20, None) == -1
    assert C.LIB.cola_checks_probe(0, 8, 1 << 20, 1024, None) == -1
    assert C.cola_strerror(-7).startswith("an index failed its bounds check")


def test_pm_path_setter_validates_without_launching():
    import paper_1509_04685_gb300 as C
    for bad in (-1, 3, 100):
        assert C.LIB.cola_pm_set_path(bad) == -1
    for good in (1, 2, 0):
        assert C.LIB.cola_pm_set_path(good) == 0


def test_pm_path_rule_without_launching():
    # automatic choice: fused where both fused z passes have warp-row forms (768,
    # 1536) and nq^3 / ng^2 <= 96; separate otherwise; a forced mode wins
    import paper_1509_04685_gb300 as C
    byref = ctypes.byref
    cases = {(512, 1536, 1536.0): 1, (256, 768, 768.0): 1, (768, 2304, 1536.0): 2, (768, 1152, 1536.0): 2,
             (384, 1152, 1152.0): 2, (256, 256, 512.0): 2, (32, 96, 128.0): 2, (1536, 1536, 1536.0): 2}
    try:
        assert C.LIB.cola_pm_set_path(0) == 0
        for (nq, ng, L), want in cases.items():
            cfg = C.make_config(nq, ng, L, 0.05)
            assert C.LIB.cola_pm_path(byref(cfg)) == want, (nq, ng)
        cfg = C.make_config(32, 96, 128.0, 0.05)
        for mode in (1, 2):
            assert C.LIB.cola_pm_set_path(mode) == 0
            assert C.LIB.cola_pm_path(byref(cfg)) == mode
        assert C.LIB.cola_pm_path(byref(C.make_config(32, 97, 128.0, 0.05))) == -3
    finally:
        C.LIB.cola_pm_set_path(0)
