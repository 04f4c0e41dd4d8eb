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
    """No kernel spills registers, except at most 16 bytes of spill stores in
    the packed kernels where that was measured faster: the global /
    semi-global inter-sequence kernels (a resident block bought by the
    occupancy table), the protein search kernel (its batch loop unrolled by
    two) and the packed long-pair kernel (semi-global, 20 columns per lane)."""
    logs = glob.glob(os.path.join(ROOT, "paper_2205_07610_gb300", "_build", "*.ptxas.txt"))
    assert logs
    text = "".join(open(f).read() for f in logs)
    assert "sm_103a" in text
    found = re.findall(r"Compiling entry function '(\S+)'.*?(\d+) bytes spill stores", text, flags=re.S)
    assert found
    for name, spill in found:
        allowed = name.startswith("_ZN2ga9ka_kernelINS_9CellS16x2ELi1") or \
            name.startswith("_ZN2ga9ka_kernelINS_9CellS16x2ELi2") or \
            name.startswith("_ZN2ga9kp_kernel") or name.startswith("_ZN2ga9kw_kernelILi2E")
        assert int(spill) <= (16 if allowed else 0), (name, spill)


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
    assert ga.Tuning((1 << 16) | 0b101, 0, 1, 0).as_dict() == {"tiles16": [6, 8, 32], "tiles32": [], "concurrent": 1,
                                                               "lanes_alt": []}
    assert ga.Tuning(0x1ff, 0, 0, 0b101).as_dict()["lanes_alt"] == [6, 8]


def test_multi_mode_arguments_rejected_before_any_cuda_call(libpath):
    """ga_align_batch_modes / ga_align_batch_host_modes check the mode list
    (1..8 entries, each local, global or semi-global) and the buffers before
    anything touches the device."""
    import numpy as np
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    sc, keep = ga.make_scoring(np.zeros((4, 4), dtype=np.int8), 5, 2)
    for fn in ("ga_align_batch_modes", "ga_align_batch_host_modes"):
        f = getattr(lib, fn)
        for modes in ([], [0] * 9, [1, 3], [-1], [2, 0, 7]):
            md = np.asarray(modes if modes else [0], dtype=np.int32)
            rc = f(None, None, None, None, 4, ctypes.byref(sc), md.ctypes.data, len(modes), None, None, None)
            assert rc == 1, (fn, modes)
        md = np.asarray([0, 1], dtype=np.int32)
        assert f(None, None, None, None, 4, ctypes.byref(sc), None, 2, None, None, None) == 1, fn  # no mode list
        assert f(None, None, None, None, 4, ctypes.byref(sc), md.ctypes.data, 2, None, None, None) == 1, fn  # no buffers
        assert f(None, None, None, None, -1, ctypes.byref(sc), md.ctypes.data, 2, None, None, None) == 1, fn
        bad, keep2 = ga.make_scoring(np.zeros((4, 4), dtype=np.int8), 2, 3)  # gap_extend > gap_open
        qo = np.zeros(2, dtype=np.int64)
        codes = np.zeros(1, dtype=np.uint8)
        sco = np.zeros(4, dtype=np.int32)
        if fn == "ga_align_batch_host_modes":
            # host buffers: the scoring is checked before any copy is made
            rc = f(codes.ctypes.data, qo.ctypes.data, codes.ctypes.data, qo.ctypes.data, 1, ctypes.byref(bad),
                   md.ctypes.data, 2, sco.ctypes.data, None, None)
            assert rc == 1, fn


def test_bad_scoring_rejected_before_any_cuda_call(libpath):
    """Every entry point that takes a scoring returns GA_ERR_ARG for an
    invalid one (gap_extend > gap_open, gap_open <= 0) synchronously, with
    non-null buffers, before any stream, copy, allocation or launch (on a
    machine without a GPU a CUDA call made first would answer GA_ERR_CUDA)."""
    import numpy as np
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    m = np.zeros((4, 4), dtype=np.int8)
    codes = np.zeros(8, dtype=np.uint8)
    off = np.array([0, 4], dtype=np.int64)
    out = np.zeros(8, dtype=np.int32)
    md = np.array([0, 1], dtype=np.int32)
    c, o, s = codes.ctypes.data, off.ctypes.data, out.ctypes.data
    for go, ge in ((2, 3), (0, 1), (5, 0)):
        sc, keep = ga.make_scoring(m, go, ge)
        r = ctypes.byref(sc)
        calls = {
            "ga_align_batch": lambda: lib.ga_align_batch(c, o, c, o, 1, r, 1, s, None, None),
            "ga_align_batch_modes": lambda: lib.ga_align_batch_modes(c, o, c, o, 1, r, md.ctypes.data, 2, s, None,
                                                                     None),
            "ga_align_batch_host": lambda: lib.ga_align_batch_host(c, o, c, o, 1, r, 1, s, None, None),
            "ga_align_batch_host_modes": lambda: lib.ga_align_batch_host_modes(c, o, c, o, 1, r, md.ctypes.data, 2,
                                                                               s, None, None),
            "ga_align_cross": lambda: lib.ga_align_cross(c, o, 1, c, o, 1, r, 0, s, None, None),
            "ga_align_long": lambda: lib.ga_align_long(c, 4, c, 4, r, 1, s, None, None),
            "ga_align_long_noalloc": lambda: lib.ga_align_long_noalloc(c, 4, c, 4, r, 1, s, None),
            "ga_align_banded": lambda: lib.ga_align_banded(c, o, c, o, 1, r, None, 16, s, None, None, None),
        }
        for name, call in calls.items():
            assert call() == 1, (name, go, ge)


def test_band_mlp_and_server_arguments_rejected_before_any_cuda_call(libpath):
    """The band-predictor, network and server entry points return GA_ERR_ARG
    for null buffers, negative sizes or an invalid scoring before anything
    touches the device."""
    import numpy as np
    import paper_2205_07610_gb300 as ga
    lib = ga.load()
    c = np.zeros(8, np.uint8)
    o = np.array([0, 4], np.int64)
    f = np.zeros(64, np.float32)
    i = np.zeros(8, np.int32)
    u = np.zeros(8, np.uint16)
    C, O, F, I, U = c.ctypes.data, o.ctypes.data, f.ctypes.data, i.ctypes.data, u.ctypes.data
    bad, keep = ga.make_scoring(np.zeros((4, 4), np.int8), 2, 3)
    fl = ctypes.c_float
    adam = (fl(1e-3), fl(0.9), fl(0.999), fl(1e-8))
    st, w = ctypes.c_int32(0), ctypes.c_int64(0)
    calls = {
        "features npairs < 0": lambda: lib.ga_band_features(C, O, C, O, -1, F, None, None),
        "features null codes": lambda: lib.ga_band_features(None, O, C, O, 1, F, None, None),
        "min_w bad scoring": lambda: lib.ga_band_min_w(C, O, C, O, 1, ctypes.byref(bad), I, I, None, None),
        "predict null params": lambda: lib.ga_band_predict(C, O, C, O, 1, None, fl(0.25), I, None, None, None),
        "predict npairs < 0": lambda: lib.ga_band_predict(C, O, C, O, -1, U, fl(0.25), I, None, None, None),
        "forward n < 0": lambda: lib.ga_mlp_forward(U, F, -1, F, None),
        "forward null params": lambda: lib.ga_mlp_forward(None, F, 1, F, None),
        "loss_grad n = 0": lambda: lib.ga_mlp_loss_grad(U, F, F, 0, F, None, None),
        "loss_grad null x": lambda: lib.ga_mlp_loss_grad(U, None, F, 1, F, None, None),
        "train steps < 0": lambda: lib.ga_mlp_train(F, U, F, F, F, F, 4, I, -1, 1, 0, *adam, None, None),
        "train batch = 0": lambda: lib.ga_mlp_train(F, U, F, F, F, F, 4, I, 1, 0, 0, *adam, None, None),
        "train null master": lambda: lib.ga_mlp_train(None, U, F, F, F, F, 4, I, 1, 1, 0, *adam, None, None),
        "cast null master": lambda: lib.ga_mlp_cast(None, U, None),
        "server_create null": lambda: lib.ga_server_create(None, None),
        "server_drain null": lambda: lib.ga_server_drain(None, 10),
        "bounded wait limit < 0": lambda: lib.ga_probe_bounded_wait(0, 1, -1, ctypes.byref(st), ctypes.byref(w)),
        "bounded wait limit > 1 s": lambda: lib.ga_probe_bounded_wait(0, 1, 2_000_000_000, ctypes.byref(st),
                                                                      ctypes.byref(w)),
        "bounded wait null out": lambda: lib.ga_probe_bounded_wait(0, 1, 1000, None, ctypes.byref(w)),
    }
    for name, call in calls.items():
        assert call() == 1, name
