"""The mechanism-specialised rates kernel's source (nk_jit_source, host only): one block of
straight-line code per reaction with the mechanism's data as literals, and it compiles with
NVRTC for sm_103a (no device needed)."""
import ctypes
import os

import pytest

import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth

NVRTC = "/usr/local/cuda/lib64/libnvrtc.so.13"


def test_source_shape(mech9):
    src = nk.jit_source(mech9)
    assert 'extern "C" __global__' in src and "nk_jit_rates" in src
    assert src.count("// reaction ") == mech9.R
    # no mechanism table is read at run time: only the math tables (gtab) and the state
    assert "DevMech" not in src and "eff_sp" not in src
    # every species row is written, with literal indices
    for k in range(mech9.K):
        assert f"omega[{k} * ld + i]" in src


def test_source_is_deterministic(mech9):
    assert nk.jit_source(mech9) == nk.jit_source(mech9.copy())


def test_too_small_buffer_is_an_error(mech9):
    d, keep = nk._desc_from(mech9)
    n = ctypes.c_size_t(16)
    buf = ctypes.create_string_buffer(16)
    assert nk.lib().nk_jit_source(ctypes.byref(d), buf, ctypes.byref(n)) != 0
    assert n.value > 16


@pytest.mark.skipif(not os.path.exists(NVRTC), reason="NVRTC not installed")
@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_source_compiles_with_nvrtc(name):
    lib = ctypes.CDLL(NVRTC)
    src = nk.jit_source(synth.mechanism(name)).encode()
    hdr = open(os.path.join(os.path.dirname(nk.__file__), "csrc", "nk_math.cuh")).read().encode()
    prog = ctypes.c_void_p()
    hs = (ctypes.c_char_p * 1)(hdr)
    hn = (ctypes.c_char_p * 1)(b"nk_math.cuh")
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), src, b"jit.cu", 1, hs, hn) == 0
    opts = (ctypes.c_char_p * 3)(b"--gpu-architecture=sm_103a", b"-std=c++17", b"--fmad=true")
    rc = lib.nvrtcCompileProgram(prog, 3, opts)
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value)
    lib.nvrtcGetProgramLog(prog, log)
    assert rc == 0, log.value.decode()
    lib.nvrtcGetCUBINSize(prog, ctypes.byref(n))
    assert n.value > 0
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
