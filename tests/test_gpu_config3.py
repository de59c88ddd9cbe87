"""The batched configuration at its full size: 24^3 x 48 (simulated lattice
48 x 24 x 24 x 24, V = 663,552), antiperiodic time, 5 stout steps, qhat = -2,
kappa = 0.136377, csw 1.90952 / 1.0.

  * 12 complex64 right-hand sides in one call of qxd_apply_Dw and of
    qxd_apply_Dhat_eo (the fused multi-right-hand-side kernel with its autotuned
    shape), FP32 and bfloat16 storage, against the oracle at sampled sites of
    every right-hand side;
  * the multi-shift CG over the ten shifts mu_j^2 of the printed degree-10
    approximation of x^(-1/4) (App. C, [Rational 0]; Sec. 4.4 MSCG) with the FP32
    Krylov space and FP64 refinement: every shift's residual
    |phi - (Dhat^+ Dhat + mu_j^2) x_j| / |phi|, evaluated by the oracle at sampled
    even sites, within 1.5e-10.

The oracle evaluates Dhat and Dhat^+ Dhat at a sample of sites from the values
on their neighbourhoods (two hops for Dhat, four for Dhat^+ Dhat), so the full
lattice never passes through it.  Tolerances are those of test_gpu_operator.py.
"""
import os

import numpy as np
import pytest

from oracle import ratapprox
from oracle.dirac import gamma5
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rational_deg10_pow_m1_4.txt")
L3 = (48, 24, 24, 24)
BF16_U = 2.0 ** -9
TOL_DW = {1: 2e-6, 2: 2 * BF16_U}
TOL_DHAT = {1: 2e-6, 2: 3 * BF16_U}


def neighbourhood(op, sites):
    """The sites one hop away from `sites` (lexicographic indices), without repeats."""
    g = op.geom
    nb = [g.neighbour(sites, mu, s)[0] for mu in range(4) for s in (+1, -1)]
    return np.unique(np.concatenate(nb))


def dhat_at(op, psi_e, sites):
    """(Dhat psi_e)(x) at the even sites x in `sites`: psi_e is an even-site field
    [V/2][4][3] (site x at position x // 2); only psi_e within two hops of `sites`
    is read.  Dhat = D_ee - D_eo D_oo^-1 D_oe (Sec. 2.3)."""
    V = op.geom.V
    full = np.zeros((V, 4, 3), dtype=np.complex128)
    ev = op.even_sites()
    full[ev] = psi_e
    odd = neighbourhood(op, sites)
    t = op.apply(full, odd)  # D_oe psi_e on the odd neighbours (full is zero on odd sites)
    Dinv = np.linalg.inv(op.diag_term(odd))
    t = np.einsum("nab,nb->na", Dinv, t.reshape(-1, 12)).reshape(-1, 4, 3)
    tf = np.zeros_like(full)
    tf[odd] = t
    return op.apply(full, sites) - op.apply(tf, sites)


def normal_at(op, x_e, sites):
    """(Dhat^+ Dhat x_e)(x) at the even sites `sites`, Dhat^+ = gamma5 Dhat gamma5."""
    near = neighbourhood(op, neighbourhood(op, sites))  # even sites within two hops
    y = np.zeros_like(x_e)
    y[near // 2] = gamma5(dhat_at(op, x_e, near))
    return gamma5(dhat_at(op, y, sites))


@pytest.fixture(scope="module")
def config3():
    import torch
    qxd, ctx, op, _, _ = setup(L3, 0, (np.pi, 0.0, 0.0, 0.0), qhat=-2, kappa=0.136377, seed=3000, stout=5,
                               device="cuda" if torch.cuda.is_available() else "cpu")
    assert op.geom.V == 663552
    yield qxd, ctx, op
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_twelve_rhs_one_launch(config3, prec):
    import torch
    qxd, ctx, op = config3
    V = op.geom.V
    nrhs = 12
    rng = np.random.default_rng(30 + prec)
    psi = torch.from_numpy(workload.spinor(V, 3010, nrhs=nrhs)).to(torch.complex64).cuda()
    out = torch.empty_like(psi)
    ctx.profile(1)
    ctx.apply_Dw(0, prec, psi, out, nrhs=nrhs)
    torch.cuda.synchronize()
    launches = {p["name"]: p["launches"] for p in ctx.profile_entries()}
    ctx.profile(0)
    # one launch per half lattice for all twelve right-hand sides
    hops = {k: v for k, v in launches.items() if k.startswith("hop_")}
    assert sum(hops.values()) == 2 and all(k.endswith("_mrhs") for k in hops), launches
    pin, pout = psi.cpu().numpy(), out.cpu().numpy()
    for r in range(nrhs):
        sites = rng.choice(V, 200, replace=False)
        ref = op.apply(pin[r].astype(np.complex128), sites)
        assert relerr(pout[r][sites].astype(np.complex128), ref) <= TOL_DW[prec], r
    del psi, out
    ne = V // 2
    pe = torch.from_numpy(workload.spinor(ne, 3011, nrhs=nrhs)).to(torch.complex64).cuda()
    oe = torch.empty_like(pe)
    ctx.apply_Dhat_eo(0, prec, pe, oe, nrhs=nrhs)
    pe_h, oe_h = pe.cpu().numpy(), oe.cpu().numpy()
    ev = op.even_sites()
    for r in range(nrhs):
        sites = ev[rng.choice(ne, 100, replace=False)]
        ref = dhat_at(op, pe_h[r].astype(np.complex128), sites)
        assert relerr(oe_h[r][sites // 2].astype(np.complex128), ref) <= TOL_DHAT[prec], r


def test_ten_shift_mscg(config3):
    import torch
    qxd, ctx, op = config3
    r = ratapprox.load(GOLDEN)
    sigma = r.mu ** 2
    assert len(sigma) == 10
    ne = op.geom.V // 2
    phi = workload.spinor(ne, 3020)
    x = torch.empty((len(sigma), ne, 4, 3), dtype=torch.complex128, device="cuda")
    info = ctx.solve_multishift(0, sigma, torch.from_numpy(phi).cuda(), x, tol=1e-10, inner=qxd.FP32)
    assert info.status == 0 and info.true_relres <= 1e-10, info.asdict()
    xs = x.cpu().numpy()
    del x
    sites = op.even_sites()[np.random.default_rng(3).choice(ne, 60, replace=False)]
    for j, s in enumerate(sigma):
        res = phi[sites // 2] - (normal_at(op, xs[j], sites) + s * xs[j][sites // 2])
        rel = float(np.linalg.norm(res) / np.linalg.norm(phi[sites // 2]))
        assert rel <= 1.5e-10, (j, s, rel)
