"""The library's host code (no GPU): the partial-fraction residues of the rational
factors and the block neighbour table of SAP and deflation, against the oracle
(oracle/ratapprox.py, oracle/reweighting.py, oracle/deflation.py), which is
pinned by its own tests."""
import os

import numpy as np
import pytest

from oracle import ratapprox
from oracle import reweighting as rw
from oracle.deflation import block_neighbours as oracle_neighbours
from oracle.sap import SAP
from tests.oracle_helpers import make_op

qxd = pytest.importorskip("paper_1908_11673_gb300.qxd")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rational_deg10_pow_m1_4.txt")


@pytest.fixture(scope="module")
def lib():
    from paper_1908_11673_gb300 import build
    build.build()
    return qxd.load_library()


def rational(r):
    return qxd.rational(r.A, r.nu, r.mu)


@pytest.mark.parametrize("k,l", [(0, 9), (0, 4), (5, 9), (3, 3)])
def test_factor_residues_match_oracle(lib, k, l):
    r = ratapprox.load(GOLDEN)
    got = qxd.rat_residues(rational(r), k, l)
    want = r.sigma(k, l)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("k,l", [(0, 9), (2, 6)])
def test_rtm_residues_match_oracle(lib, k, l):
    r_t = ratapprox.load(GOLDEN)
    r_mu = rw.shifted(r_t, 0.02)
    s1, s2 = qxd.rtm_residues(rational(r_mu), rational(r_t), k, l)
    w1, w2 = rw.rtm_sigma(r_mu, r_t, k, l)
    assert np.abs(s1 - w1).max() <= 1e-12 * np.abs(w1).max()
    assert np.abs(s2 - w2).max() <= 1e-12 * np.abs(w2).max()


def test_residue_errors(lib):
    same = qxd.rational(1.0, [1.0, 2.0], [0.5, 0.5])
    with pytest.raises(qxd.QxdError):
        qxd.rat_residues(same, 0, 1)
    r = rational(ratapprox.load(GOLDEN))
    with pytest.raises(qxd.QxdError):
        qxd.rat_residues(r, 4, 2)


@pytest.mark.parametrize("L,cstar", [((8, 8, 8, 8), 0), ((16, 8, 8, 8), 0), ((8, 4, 8, 8), 1), ((8, 4, 8, 8), 3)])
def test_block_neighbours_match_oracle(lib, L, cstar):
    op, _, _ = make_op(L, cstar, (np.pi, 0, 0, 0), seed=5)
    want = oracle_neighbours(SAP(op, bsize=4), op.geom)
    got = qxd.block_neighbours(L, cstar)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("L", [(12, 8, 8, 8), (8, 8, 4, 8), (7, 8, 8, 8)])
def test_block_neighbours_rejects(lib, L):
    with pytest.raises(qxd.QxdError):
        qxd.block_neighbours(L)


def test_geometry_validation_of_the_time_boundary(lib):
    """qxd_create checks the geometry before it touches a device: an open time
    boundary with a time phase, an unknown boundary type and a non-finite cF are
    refused with QXD_EARG."""
    for theta, tbc, cF in (((np.pi, 0, 0, 0), qxd.TBC_OPEN, 1.0), ((0, 0, 0, 0), 2, 1.0),
                           ((0, 0, 0, 0), qxd.TBC_OPEN, float("nan"))):
        with pytest.raises(qxd.QxdError) as e:
            qxd.Context((4, 4, 4, 4), 0, theta, tbc=tbc, cF=cF)
        assert e.value.code == 1
