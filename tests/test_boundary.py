"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ga_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    import paper_2205_07610_gb300 as ga
    return ga.build()


def test_header_declares_the_binding_surface():
    import paper_2205_07610_gb300 as ga
    assert _declared() == set(ga.EXPORTED)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ga_[a-z0-9_]+)$", out, flags=re.M))
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    for name in ga.EXPORTED:
        assert hasattr(lib, name)
    assert ga.version() >= 100
    assert ga.strerror(5) == "residue code outside the alphabet"
    assert ga.strerror(0) == "ok"


def test_kernels_compiled_for_sm103a_without_spills(libpath):
    """No kernel spills registers, except the packed global / semi-global
    inter-sequence kernels, whose occupancy table allows at most 16 bytes of
    spill stores where that bought a resident block."""
    logs = glob.glob(os.path.join(ROOT, "paper_2205_07610_gb300", "_build", "*.ptxas.txt"))
    assert logs
    text = "".join(open(f).read() for f in logs)
    assert "sm_103a" in text
    found = re.findall(r"Compiling entry function '(\S+)'.*?(\d+) bytes spill stores", text, flags=re.S)
    assert found
    for name, spill in found:
        packed_gs = name.startswith("_ZN2ga9ka_kernelINS_9CellS16x2ELi1") or \
            name.startswith("_ZN2ga9ka_kernelINS_9CellS16x2ELi2")
        assert int(spill) <= (16 if packed_gs else 0), (name, spill)


def test_argument_errors_are_synchronous(libpath):
    """Invalid scoring is rejected before anything touches the device."""
    import numpy as np
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    m = np.zeros((4, 4), dtype=np.int8)
    for go, ge, want in ((0, 1, 1), (2, 3, 1), (5, 0, 1)):
        sc, keep = ga.make_scoring(m, go, ge)
        rc = lib.ga_align_batch(None, None, None, None, 0, ctypes.byref(sc), 0, None, None, None)
        assert rc == want
    sc, keep = ga.make_scoring(np.zeros((40, 40), np.int8), 5, 2)
    assert lib.ga_align_batch(None, None, None, None, 0, ctypes.byref(sc), 0, None, None, None) == 2
    sc, keep = ga.make_scoring(m, 5, 2)
    assert lib.ga_align_batch(None, None, None, None, 0, ctypes.byref(sc), 7, None, None, None) == 1
    assert lib.ga_align_batch(None, None, None, None, -1, ctypes.byref(sc), 0, None, None, None) == 1


def test_plan_arguments_rejected_before_any_cuda_call(libpath):
    """Batch-plan argument errors are returned before the device is touched."""
    import numpy as np
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    m = np.zeros((4, 4), dtype=np.int8)
    sc, keep = ga.make_scoring(m, 5, 2)
    h = ctypes.c_void_p()
    # bad mode, max_pairs < 1, negative residues, max_len < 1, null out pointer
    for mode, mp, mr, ml in ((3, 10, 10, 10), (0, 0, 10, 10), (0, 10, -1, 10), (0, 10, 10, 0)):
        assert lib.ga_plan_create(ctypes.byref(sc), mode, mp, mr, ml, ctypes.byref(h)) == 1
    assert lib.ga_plan_create(ctypes.byref(sc), 0, 10, 10, 10, None) == 1
    bad, keep2 = ga.make_scoring(m, 2, 3)  # gap_extend > gap_open
    assert lib.ga_plan_create(ctypes.byref(bad), 0, 10, 10, 10, ctypes.byref(h)) == 1
    tu = ga.Tuning(0x1ff, 0x1ff, 0, 0)
    for fn, args in (("ga_plan_run", (None, None, None, None, None, 0, None, None)),
                     ("ga_plan_capture", (None, None, None, None, None, 0, None)),
                     ("ga_plan_launch", (None, None)),
                     ("ga_plan_stats", (None, None, None)),
                     ("ga_plan_get_tuning", (None, ctypes.byref(tu))),
                     ("ga_plan_set_tuning", (None, ctypes.byref(tu))),
                     ("ga_plan_destroy", (None,))):
        assert getattr(lib, fn)(*args) == 1, fn
    assert ctypes.sizeof(ga.Tuning) == 16
    assert ga.Tuning((1 << 16) | 0b101, 0, 1, 0).as_dict() == {"tiles16": [6, 8, 32], "tiles32": [], "concurrent": 1}
