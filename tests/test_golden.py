"""The stored fixture under tests/golden/ (CPU only).

tiny_pair.txt holds oracle values on a hand-written 7-node instance,
written by tests/golden/make_golden.py from the oracle alone.  The oracle
must keep reproducing them (a change to its arithmetic regenerates the
file, with the passage that justifies it in the commit message), and the
values carry properties fixed by the instance itself: the planted
relabelling is what the final plan's top-1 recovers, and every row of a
plan ends exactly on its marginal (Eq. 3 ends on the row update).
"""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _stored(m):
    return m.parse(open(os.path.join(HERE, "golden", "tiny_pair.txt")).read())


def test_oracle_reproduces_the_fixture():
    m = _maker()
    want, got = _stored(m), m.compute()
    np.testing.assert_allclose(got["C_node"], want["C_node"], rtol=1e-12, atol=0)
    for k in ("logS_1", "logS_3"):
        np.testing.assert_allclose(got[k], want[k], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(got["top1"], want["top1"])


def test_fixture_properties_fixed_by_the_instance():
    m = _maker()
    v = _stored(m)
    np.testing.assert_array_equal(v["top1"], m.PERM)          # the planted relabelling
    for k in ("logS_1", "logS_3"):
        S = np.exp(v[k])
        np.testing.assert_allclose(S.sum(axis=1), 1.0 / m.N, rtol=1e-12)
        # 30 iterations leave the columns a few 1e-3 off in L1
        assert np.abs(S.sum(axis=0) - 1.0 / m.N).sum() < 1e-2
    assert v["C_node"].shape == (m.N, m.N) and np.all(v["C_node"] > 0)


def test_render_and_parse_round_trip():
    m = _maker()
    v = m.compute()
    back = m.parse(m.render(v))
    for k in v:
        np.testing.assert_array_equal(back[k], v[k])
