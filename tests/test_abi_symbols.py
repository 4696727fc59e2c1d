"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(hfmm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2006_14952_gb300 import build, hfmm

    path = build.build()
    lib = ctypes.CDLL(path)
    decl = declared_functions()
    assert len(decl) >= 9
    missing = [s for s in decl if not hasattr(lib, s)]
    assert not missing, missing
    assert set(hfmm.SYMBOLS) <= set(decl)


def test_parameter_validation_needs_no_gpu():
    from paper_2006_14952_gb300 import hfmm

    L = hfmm.load()
    p = hfmm.default_params()
    assert p.order == 4 and p.leaf_max == 16 and p.transition_rule == 1 and p.size_rule == 1
    h = ctypes.c_void_p()
    p.order = 99
    assert L.hfmm_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert b"order" in L.hfmm_last_error(None)
    p.order = 4
    p.rcut_rs = 1000.0
    assert L.hfmm_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert L.hfmm_create(None, ctypes.byref(h)) == -1
    # the tree choice: 0 or 1, and the k-d tree only with the options it supports
    p = hfmm.default_params()
    assert p.tree == 0
    p.tree = 2
    assert L.hfmm_create(ctypes.byref(p), ctypes.byref(h)) == -1 and b"tree" in L.hfmm_last_error(None)
    for field, value in (("mac_mode", 1), ("m2l_precision", 1), ("m2l_tables", 1), ("order", 7)):
        p = hfmm.default_params()
        p.tree = 1
        setattr(p, field, value)
        assert L.hfmm_create(ctypes.byref(p), ctypes.byref(h)) == -1
        assert b"tree 1" in L.hfmm_last_error(None), field


def test_struct_layout_matches_header():
    """The ctypes mirrors have the sizes the C compiler gives the header structs."""
    import subprocess
    import tempfile

    from paper_2006_14952_gb300 import hfmm

    src = '#include <stdio.h>\n#include "hfmm.h"\nint main(){printf("%zu %zu\\n", sizeof(hfmm_params), sizeof(hfmm_stats));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        a, b = map(int, subprocess.check_output([exe]).split())
    assert a == ctypes.sizeof(hfmm.Params) and b == ctypes.sizeof(hfmm.Stats)


def test_every_context_call_rejects_a_null_context_without_a_gpu():
    """A NULL context is an argument error before any CUDA call is made."""
    from paper_2006_14952_gb300 import hfmm

    L = hfmm.load()
    out = (ctypes.c_int64 * 4)()
    nb = ctypes.c_size_t(0)
    cnt = ctypes.c_int64(0)
    calls = {
        "hfmm_build_tree": lambda: L.hfmm_build_tree(None, None, None, 0, None),
        "hfmm_short_range_forces": lambda: L.hfmm_short_range_forces(None, None, None),
        "hfmm_short_range_forces_host": lambda: L.hfmm_short_range_forces_host(None, None, None, 0, None, None),
        "hfmm_pm_long_range": lambda: L.hfmm_pm_long_range(None, None, None),
        "hfmm_step": lambda: L.hfmm_step(None, None, None, None, 0.0, None),
        "hfmm_interaction_counts": lambda: L.hfmm_interaction_counts(None, 0, out, None),
        "hfmm_get_stats": lambda: L.hfmm_get_stats(None, None),
        "hfmm_export": lambda: L.hfmm_export(None, 0, None, ctypes.byref(nb)),
        "hfmm_load_mlp": lambda: L.hfmm_load_mlp(None, None, 0),
        "hfmm_collect_training_pairs": lambda: L.hfmm_collect_training_pairs(None, 1, 1, None, None,
                                                                             ctypes.byref(cnt), None),
    }
    for name, call in calls.items():
        assert call() == -1, name  # HFMM_ERR_ARG
    L.hfmm_destroy(None)  # accepted
    assert L.hfmm_last_error(None) is not None


def test_alu_probe_rejects_bad_arguments_without_a_gpu():
    from paper_2006_14952_gb300 import hfmm

    L = hfmm.load()
    rate = ctypes.c_double(0.0)
    assert L.hfmm_alu_peak(4, 1, None, ctypes.byref(rate), None, None) == -1
    assert L.hfmm_alu_peak(0, 0, None, ctypes.byref(rate), None, None) == -1
    assert L.hfmm_alu_peak(0, 1, None, None, None, None) == -1
