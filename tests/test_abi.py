"""The C-ABI library builds, loads and exports every entry point of include/nkchem.h; its
host-side argument checks run without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import build as nkbuild
from paper_2409_06404_gb300 import synth
from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "nkchem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nk_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    nkbuild.build()
    return nk.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("nk_mechanism_load", "nk_mechanism_free", "nk_thermo_eval", "nk_rates_eval", "nk_transport_eval",
              "nk_rates_jvp", "nk_rates_vjp", "nk_rates_vjp_workspace", "nk_last_error", "nk_version"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", nk.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (nk_\w+)", out))
    for f in declared_functions():
        assert f in exported, f
        assert hasattr(lib, f)


def test_build_targets_sm_103a_only():
    assert nkbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_error_string(lib):
    assert lib.nk_version() == 1
    assert isinstance(lib.nk_last_error(), bytes)


def test_null_mechanism_is_rejected(lib):
    st = lib.nk_rates_eval(None, 10, 10, None, None, None, None, None, None, 0, None)
    assert st == 1 and b"mech" in lib.nk_last_error()
    st = lib.nk_transport_eval(None, 10, 10, None, None, None, None, None, None, 0, None)
    assert st == 1
    st = lib.nk_mechanism_info(None, None, None)
    assert st == 1


def test_null_mechanism_is_rejected_by_every_point_entry(lib):
    """Each entry that takes a mechanism returns NK_EINVAL for NULL before touching the device
    (the single-precision linearization, its products, the reactor, the Jacobian and
    block-Jacobi entries, the host-resident evaluation)."""
    calls = {
        "nk_rates_linearize": (None, 8, 8, None, None, None, None, None, 8, None),
        "nk_rates_jvp_linearized": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None),
        "nk_rates_linearize_f32": (None, 8, 8, None, None, None, None, None, 8, None),
        "nk_rates_jvp_linearized_f32": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None),
        "nk_rhs_jvp_linearized": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None, None, None),
        "nk_rhs_jvp_linearized_f32": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None, None,
                                      None),
        "nk_rhs_jacobian": (None, 8, 8, None, None, None, None, 8, None, None, None, 8, None),
        "nk_rates_linearize_compact": (None, 8, 8, None, None, None, None, None, 8, None, None, None),
        "nk_rates_jvp_linearized_compact": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None),
        "nk_rhs_jvp_linearized_compact": (None, 8, 8, None, None, None, None, 8, None, None, None, None, None, None,
                                          None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == 1, name
        assert b"NULL" in lib.nk_last_error() or b"mech" in lib.nk_last_error(), name
    slots = ctypes.c_int64()
    assert lib.nk_rates_linearization_slots(None, ctypes.byref(slots)) == 1
    assert lib.nk_rates_linearization_slots_f32(None, ctypes.byref(slots)) == 1
    assert lib.nk_rates_linearization_slots_compact(None, ctypes.byref(slots)) == 1
    b = ctypes.c_size_t()
    o = nk.reactor_opts(linearized=2)
    assert lib.nk_reactor_workspace(None, 8, ctypes.byref(o), ctypes.byref(b)) == 1


def _desc(mech):
    d, keep = nk._desc_from(mech)
    return d, keep


def _load_status(lib, mech):
    d, keep = _desc(mech)
    h = ctypes.c_void_p()
    st = lib.nk_mechanism_load(ctypes.byref(d), ctypes.byref(h))
    msg = lib.nk_last_error().decode()
    if st == 0:
        lib.nk_mechanism_free(h)
    return st, msg


def test_mechanism_descriptor_checks(lib, mech9):
    bad = mech9.copy()
    bad.reac_sp = bad.reac_sp.copy()
    bad.reac_sp[0] = 99
    st, msg = _load_status(lib, bad)
    assert st == 1 and "out of range" in msg
    bad = mech9.copy()
    bad.rtype = bad.rtype.copy()
    bad.rtype[0] = 7
    assert _load_status(lib, bad)[0] == 1
    bad = mech9.copy()
    bad.W = bad.W.copy()
    bad.W[2] = -1.0
    assert _load_status(lib, bad)[0] == 1
    bad = mech9.copy()
    bad.reac_nu = bad.reac_nu.copy()
    bad.reac_nu[0] = 9
    assert _load_status(lib, bad)[0] == 5          # NK_EUNSUPPORTED
    bad = mech9.copy()
    bad.troe = bad.troe.copy()
    r = int(np.flatnonzero(bad.rtype == 2)[0])
    bad.troe[r, 1] = 0.0
    assert _load_status(lib, bad)[0] == 1


def test_valid_descriptor_without_gpu_reports_cuda_error(lib, mech9):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, msg = _load_status(lib, mech9)
    assert st == 3, msg                            # NK_ECUDA, never a crash


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(nk, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nk, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        nk.lib()
