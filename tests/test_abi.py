"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function include/picount.h declares."""
import os
import re
import subprocess

import pytest

import paper_1503_01839_gb300 as pc
from paper_1503_01839_gb300 import build as pcbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "picount.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return pcbuild.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("pc_pi_count", "pc_phi", "pc_s2_hard", "pc_p2", "pc_pi_count_batch", "pc_create", "pc_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert sorted(pc.SYMBOLS) == declared_functions()


def test_library_loads_and_answers_host_calls(libpath):
    L = pc.lib()
    assert b"sm_103a" in L.pc_version()
    assert L.pc_strerror(0) == b"ok"
    assert L.pc_strerror(-2).startswith(b"x out of range")


def test_library_is_built_for_sm_103a_only():
    assert pcbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pc.PicountError):
        pc.Context(0)


def test_bad_params_rejected_before_device_work(libpath):
    for bad in ({"seg_bytes": 5120}, {"batch_launch": 2}, {"p2_bucket": 2}, {"m_source": 2}, {"pi_gather": 2}):
        with pytest.raises(pc.PicountError) as e:
            pc.Context(0, **bad)
        assert e.value.code == -1, bad
