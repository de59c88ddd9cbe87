"""Pins of the deflation oracle (oracle/deflation.py) by what the construction
fixes independently of its code:

 * the block pieces of the subspace are orthonormal (P^+ P = 1);
 * A = P^+ D P couples a block only to itself and to the blocks across its
   eight faces (the block neighbour map, C* shifts included);
 * the coarse correction makes the residual orthogonal to the subspace,
   P^+ (1 - D P A^-1 P^+) = 0, and annihilates D on it, (1 - D P A^-1 P^+) D P = 0;
 * with one-site blocks and Ns = 12 the subspace is the whole space, so M_dfl
   is D^-1 exactly (LAPACK solve);
 * gauge covariance: rotating the gauge field and the generating random fields
   rotates the preconditioner, M'[g v] = g M[v].
"""
import numpy as np
import pytest

from oracle import DiracOperator, GaugeField
from oracle.deflation import Deflation, block_neighbours
from oracle.sap import SAP
from paper_1908_11673_gb300 import workload
from tests.oracle_helpers import dense, make_op


def seeds(V, Ns, seed):
    return np.stack([workload.spinor(V, seed + k) for k in range(Ns)])


CASES = [((8, 8, 4, 4), 0, 2, 4), ((4, 4, 4, 8), 1, 2, 3)]  # L, cstar, SAP block, Ns


@pytest.fixture(scope="module", params=CASES, ids=["8x8x4x4", "cstar1_4x4x4x8"])
def dfl(request):
    L, cstar, b, Ns = request.param
    op, _, _ = make_op(L, cstar, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=211)
    sap = SAP(op, bsize=b, ncy=2, nmr=3)
    return Deflation(op, sap, seeds(op.geom.V, Ns, 212), ninv=1)


def test_block_orthonormality(dfl):
    for j in range(dfl.Ns):
        for k in range(dfl.Ns):
            d = dfl.block_dot(dfl.phis[j], dfl.phis[k])
            assert np.abs(d - (j == k)).max() < 1e-12
    c = np.random.default_rng(1).normal(size=(dfl.nblocks, dfl.Ns)) + 0j
    assert np.abs(dfl.restrict(dfl.prolong(c)) - c).max() < 1e-12


def test_little_operator_is_nearest_neighbour(dfl):
    nb = block_neighbours(dfl.sap, dfl.geom)
    Ns = dfl.Ns
    for B in range(dfl.nblocks):
        allowed = set(nb[B])
        for Bp in range(dfl.nblocks):
            blk = dfl.A[B * Ns:(B + 1) * Ns, Bp * Ns:(Bp + 1) * Ns]
            if Bp in allowed:
                assert np.abs(blk).max() > 0
            else:
                assert np.abs(blk).max() == 0.0


def test_coarse_correction_projects(dfl):
    op = dfl.op
    v = workload.spinor(dfl.geom.V, 213)
    r = v - op.apply(dfl.coarse_solve(v))
    assert np.abs(dfl.restrict(r)).max() < 1e-11 * np.abs(dfl.restrict(v)).max()
    c = np.random.default_rng(2).normal(size=(dfl.nblocks, dfl.Ns)) + 0j
    w = op.apply(dfl.prolong(c))
    assert np.linalg.norm(w - op.apply(dfl.coarse_solve(w))) < 1e-11 * np.linalg.norm(w)


def test_full_subspace_gives_the_exact_inverse():
    op, _, _ = make_op((4, 2, 2, 2), 0, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=214)
    V = op.geom.V
    sap = SAP(op, bsize=1, ncy=1, nmr=2)
    d = Deflation(op, sap, seeds(V, 12, 215), ninv=1)
    v = workload.spinor(V, 216)
    D = dense(lambda x: op.apply(x), V * 12, (V, 4, 3))
    x = np.linalg.solve(D, v.reshape(-1)).reshape(V, 4, 3)
    assert np.linalg.norm(d.apply(v) - x) < 1e-10 * np.linalg.norm(x)


def test_deflation_is_gauge_covariant():
    from tests.test_oracle_symmetries import random_su3
    qhat = -2
    op, U, A = make_op((8, 4, 4, 4), 0, (np.pi, 0, 0, 0), qhat=qhat, seed=217, kappa=0.13)
    geom = op.geom
    rng = np.random.default_rng(3)
    g = random_su3(rng, geom.V)
    lam = rng.uniform(-np.pi, np.pi, geom.V)
    s = geom.sites()
    Un, An = np.empty_like(U), np.empty_like(A)
    for mu in range(4):
        nb, _ = geom.neighbour(s, mu, +1)
        Un[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[nb], -1, -2))
        An[:, mu] = lam + A[:, mu] - lam[nb]
    op2 = DiracOperator(GaugeField(geom, Un, An, 6.0), op.fl)
    omega = g * np.exp(1j * qhat * lam)[:, None, None]
    rot = lambda v: np.einsum('nij,naj->nai', omega, v)
    sd = seeds(geom.V, 3, 218)
    d1 = Deflation(op, SAP(op, bsize=2, ncy=1, nmr=2), sd, ninv=1)
    d2 = Deflation(op2, SAP(op2, bsize=2, ncy=1, nmr=2), np.array([rot(x) for x in sd]), ninv=1)
    v = workload.spinor(geom.V, 219)
    assert np.abs(d2.apply(rot(v)) - rot(d1.apply(v))).max() < 1e-10 * np.abs(d1.apply(v)).max()
