"""The alignment server's arena bookkeeping (csrc/ga_arena.h), on the CPU:
tests/arena_check.cpp admits and completes requests of the serving length
mix in random order against the first-fit arena and the code slabs, and
checks that live ranges never overlap, that codes admitted back to back in
one slab are contiguous (one copy per scheduler tick), that an empty server
admits any request that fits its arena, and that the whole arena is free
once every request has completed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_and_code_slabs(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "arena_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", "-o", str(exe),
                    os.path.join(ROOT, "tests", "arena_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("requests admitted") == 4
