"""Pins of the SAP oracle (oracle/sap.py)."""
import numpy as np
import pytest

from oracle.sap import SAP
from paper_1908_11673_gb300 import workload
from tests.oracle_helpers import dense, make_op


def block_matrix_dense(op, sap):
    """Dense D with every entry between sites of different blocks removed."""
    V = op.geom.V
    D = dense(lambda v: op.apply(v), V * 12, (V, 4, 3))
    blk = np.repeat(sap.block, 12)
    return D * (blk[:, None] == blk[None, :])


@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), 0), ((4, 2, 4, 4), 1)])
def test_block_operator_is_D_without_cross_block_hops(L, cstar):
    op, _, _ = make_op(L, cstar, (np.pi, 0, 0, 0), qhat=4, seed=12, kappa=0.13)
    sap = SAP(op, bsize=2)
    DB = block_matrix_dense(op, sap)
    V = op.geom.V
    v = workload.spinor(V, 1)
    got = sap.mul_diag(sap.diag, v, 0) + sap.mul_diag(sap.diag, v, 1) + sap.hop_block(v, 0) + sap.hop_block(v, 1)
    assert np.abs(got.reshape(-1) - DB @ v.reshape(-1)).max() < 1e-13 * np.abs(got).max()


def test_block_minres_converges_to_the_block_inverse():
    op, _, _ = make_op((4, 4, 4, 4), 0, (np.pi, 0, 0, 0), qhat=-2, seed=13, kappa=0.125)
    sap = SAP(op, bsize=2, nmr=200)
    DB = block_matrix_dense(op, sap)
    rho = workload.spinor(op.geom.V, 2)
    for colour in (0, 1):
        d = sap.block_solve(rho, colour)
        sel = np.repeat(sap.colour == colour, 12)
        ref = np.linalg.solve(DB, np.where(sel, rho.reshape(-1), 0.0))
        ref = np.where(sel, ref, 0.0)
        assert np.linalg.norm(d.reshape(-1) - ref) < 1e-10 * np.linalg.norm(ref)


def test_sap_iteration_converges_to_the_solution():
    op, _, _ = make_op((4, 4, 4, 4), 0, (np.pi, 0, 0, 0), qhat=-2, seed=14, kappa=0.12)
    V = op.geom.V
    eta = workload.spinor(V, 3)
    D = dense(lambda v: op.apply(v), V * 12, (V, 4, 3))
    x = np.linalg.solve(D, eta.reshape(-1)).reshape(V, 4, 3)
    errs = [np.linalg.norm(SAP(op, bsize=2, ncy=c, nmr=8).apply(eta) - x) / np.linalg.norm(x) for c in (1, 3, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs


@pytest.mark.parametrize("L,b", [((2, 4, 4, 4), 2), ((4, 4, 6, 4), 2), ((4, 4, 6, 4), 4)])
def test_sap_needs_an_even_number_of_blocks(L, b):
    """one block, three blocks, and an extent that is no multiple of the block size"""
    op, _, _ = make_op(L, 0, (np.pi, 0, 0, 0))
    with pytest.raises(ValueError):
        SAP(op, bsize=b)


def test_sap_is_gauge_covariant():
    from oracle import DiracOperator, GaugeField
    from tests.test_oracle_symmetries import random_su3
    qhat = 4
    op, U, A = make_op((4, 4, 4, 4), 0, (np.pi, 0, 0, 0), qhat=qhat, seed=15)
    geom = op.geom
    rng = np.random.default_rng(1)
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
    eta = workload.spinor(geom.V, 4)
    got = SAP(op2, bsize=2, ncy=2, nmr=3).apply(rot(eta))
    want = rot(SAP(op, bsize=2, ncy=2, nmr=3).apply(eta))
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
