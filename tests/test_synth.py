"""Generator invariants: balanced reactions, well-formed tables, reproducible states."""
import numpy as np

from paper_2409_06404_gb300 import synth
from conftest import nu_matrix


def test_reactions_are_element_balanced(mech9, mech53, mech120):
    for m in (mech9, mech53, mech120):
        nu = nu_matrix(m)
        assert np.all(m.atoms.T @ nu == 0)
        # mass balance follows from atom balance
        assert np.max(np.abs(m.W @ nu)) < 1e-15


def test_table_shapes_and_types(mech53):
    m = mech53
    assert m.K == 53 and m.R == 325
    assert np.sum(m.rtype == 1) == 20 and np.sum(m.rtype == 2) == 25
    assert m.reac_ptr[0] == 0 and m.reac_ptr[-1] == len(m.reac_sp)
    assert np.all(np.diff(m.reac_ptr) >= 1) and np.all(np.diff(m.prod_ptr) >= 1)
    assert np.all(m.reac_nu >= 1) and np.all(m.prod_nu >= 1)
    assert m.D_fit.shape == (53 * 52 // 2, 4)
    assert np.all(m.troe[m.rtype != 2] == 0)
    assert np.all((m.troe[m.rtype == 2, 0] >= 0.1) & (m.troe[m.rtype == 2, 0] <= 0.9))
    assert np.all(m.eff[m.rtype == 0] == 1.0)
    A = np.exp(m.lnA)
    assert A.min() >= 1e6 * (1 - 1e-12) and A.max() <= 1e16 * (1 + 1e-12)


def test_no_duplicate_reactions(mech53):
    m = mech53
    seen = set()
    for r in range(m.R):
        a = tuple(sorted((int(m.reac_sp[i]), int(m.reac_nu[i])) for i in range(m.reac_ptr[r], m.reac_ptr[r + 1])))
        b = tuple(sorted((int(m.prod_sp[i]), int(m.prod_nu[i])) for i in range(m.prod_ptr[r], m.prod_ptr[r + 1])))
        key = tuple(sorted([a, b]))
        assert key not in seen
        seen.add(key)


def test_deterministic_in_seed():
    a = synth.make_mechanism(**synth.MECHS["h2_9sp_21rx"])
    b = synth.make_mechanism(**synth.MECHS["h2_9sp_21rx"])
    for k, v in a.arrays().items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, getattr(b, k)), k


def test_gll_nodes():
    x = synth.gll_nodes(7)
    assert x.shape == (8,)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15)
    # GLL quadrature with these nodes integrates degree <= 2p-1 = 13 exactly: check via the
    # weights w_i = 2/(p(p+1) P_p(x_i)^2) on [-1, 1]
    from numpy.polynomial import legendre as L
    t = 2 * x - 1
    w = 2.0 / (7 * 8 * L.legval(t, [0] * 7 + [1]) ** 2)
    assert abs(np.sum(w * t ** 12) - 2.0 / 13) < 1e-13


def test_states():
    st = synth.states_uniform(9, 1000, seed=3)
    assert np.allclose(st.Y.sum(axis=0), 1.0, atol=1e-14)
    assert st.T.min() >= 300 and st.T.max() <= 2500
    fl = synth.states_flame(5, 8, seed=4)
    assert fl.n == 8 * 512
    assert fl.T.min() >= 300 and fl.T.max() <= 3500
    assert np.allclose(fl.Y.sum(axis=0), 1.0, atol=1e-14)
