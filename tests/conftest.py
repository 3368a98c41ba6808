import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2409_06404_gb300 import synth  # noqa: E402

R_GAS = 8.314462618
P_ATM = 101325.0


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def mech9():
    return synth.mechanism("h2_9sp_21rx")


@pytest.fixture(scope="session")
def mech53():
    return synth.mechanism("ch4_53sp_325rx")


@pytest.fixture(scope="session")
def mech120():
    return synth.mechanism("big_120sp_700rx")


def nu_matrix(mech):
    """Net stoichiometric matrix nu[k, r] = nu''_kr - nu'_kr (test helper)."""
    nu = np.zeros((mech.K, mech.R))
    for r in range(mech.R):
        for i in range(mech.reac_ptr[r], mech.reac_ptr[r + 1]):
            nu[mech.reac_sp[i], r] -= mech.reac_nu[i]
        for i in range(mech.prod_ptr[r], mech.prod_ptr[r + 1]):
            nu[mech.prod_sp[i], r] += mech.prod_nu[i]
    return nu


# ---------------------------------------------------------------------- GPU helpers
_LOADED = {}


def gpu_mechanism(name_or_mech):
    """Library handle for a named generator mechanism (cached per session) or a Mechanism."""
    import paper_2409_06404_gb300 as nk
    if isinstance(name_or_mech, str):
        if name_or_mech not in _LOADED:
            _LOADED[name_or_mech] = nk.mechanism_load(synth.mechanism(name_or_mech))
        return _LOADED[name_or_mech]
    return nk.mechanism_load(name_or_mech)


def to_dev(*arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def host(t):
    return t.detach().cpu().numpy()


def scaled_err(actual, expect, scale):
    """max over entries of |actual - expect| / scale (0/0 counts as 0, x/0 as inf)."""
    d = np.abs(np.asarray(actual) - np.asarray(expect))
    s = np.asarray(scale, dtype=float)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(d == 0, 0.0, d / s)
    return float(np.max(r)) if r.size else 0.0


@pytest.fixture(scope="session")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return torch.device("cuda:0")
