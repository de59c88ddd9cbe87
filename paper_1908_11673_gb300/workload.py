"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the Dirac operator or of its solvers: it only
draws random gauge fields and sources and, for the smeared workloads, applies
stout smearing (a workload recipe, not part of the method).  Both sides of every
parity test receive the bytes it produces.

Recipe (all FP64, NumPy PCG64 streams):
  * SU(3) links U = exp(iH), H traceless Hermitian.  Before the trace is removed
    the diagonal entries and the real and imaginary parts of the upper
    off-diagonal entries are independent N(0, sigma_h^2).
  * U(1) angles A_mu(x) ~ N(0, sigma_a^2) (the compact field z = exp(iA) of Sec. 2).
  * Optional stout smearing of the SU(3) links (Morningstar-Peardon, isotropic,
    staples from all nu != mu, parameter rho) with periodic identification of the
    physical lattice.
  * Optional stout smearing of the U(1) links, the abelian case of the same
    recipe: z(x,mu) <- exp(i rho Im[C(x,mu) z(x,mu)^*]) z(x,mu) with C the sum of
    the six staples, i.e. A_mu(x) <- A_mu(x) + rho sum_staples sin(theta_staple - A_mu(x)),
    all directions updated at once.  Off by default (u1_stout_steps = 0).
  * Sources: complex Gaussian, real and imaginary parts N(0, 1).

Field layout: physical lattice, lexicographic site index with x0 (time) slowest,
  idx = ((x0*L1 + x1)*L2 + x2)*L3 + x3;
  U: complex128 [V][4][3][3] (row, column), A: float64 [V][4].
"""
from __future__ import annotations

import numpy as np
import torch


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_hermitian(rng: np.random.Generator, n: int, sigma: float) -> np.ndarray:
    """n traceless Hermitian 3x3 matrices, complex128 [n][3][3]."""
    h = np.zeros((n, 3, 3), dtype=np.complex128)
    d = rng.normal(0.0, sigma, size=(n, 3))
    off = rng.normal(0.0, sigma, size=(n, 3, 2))
    for i in range(3):
        h[:, i, i] = d[:, i]
    for k, (i, j) in enumerate(((0, 1), (0, 2), (1, 2))):
        h[:, i, j] = off[:, k, 0] + 1j * off[:, k, 1]
        h[:, j, i] = off[:, k, 0] - 1j * off[:, k, 1]
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    for i in range(3):
        h[:, i, i] -= tr
    return h


def _expm_i(h: torch.Tensor) -> torch.Tensor:
    """exp(i h) for a batch of Hermitian matrices (torch's matrix exponential)."""
    return torch.linalg.matrix_exp(1j * h)


def _stout_step(U: torch.Tensor, L, rho: float) -> torch.Tensor:
    """One isotropic stout-smearing step on U [L0,L1,L2,L3,4,3,3] (periodic)."""
    dag = lambda m: m.conj().transpose(-1, -2)
    new = torch.empty_like(U)
    for mu in range(4):
        C = torch.zeros_like(U[..., mu, :, :])
        Umu = U[..., mu, :, :]
        for nu in range(4):
            if nu == mu:
                continue
            Unu = U[..., nu, :, :]
            Umu_xpnu = torch.roll(Umu, -1, dims=nu)
            Unu_xpmu = torch.roll(Unu, -1, dims=mu)
            C = C + Unu @ Umu_xpnu @ dag(Unu_xpmu)
            Unu_xmnu = torch.roll(Unu, 1, dims=nu)
            Umu_xmnu = torch.roll(Umu, 1, dims=nu)
            Unu_xmnu_pmu = torch.roll(Unu_xmnu, -1, dims=mu)
            C = C + dag(Unu_xmnu) @ Umu_xmnu @ Unu_xmnu_pmu
        Om = rho * C @ dag(Umu)
        X = dag(Om) - Om
        tr = torch.diagonal(X, dim1=-2, dim2=-1).sum(-1)[..., None, None]
        eye = torch.eye(3, dtype=U.dtype, device=U.device)
        Q = 0.5j * X - (1j / 6.0) * tr * eye
        new[..., mu, :, :] = _expm_i(Q) @ Umu
    return new


def _u1_stout_step(A: torch.Tensor, rho: float) -> torch.Tensor:
    """One abelian stout step on the angles A [L0,L1,L2,L3,4] (periodic)."""
    new = torch.empty_like(A)
    for mu in range(4):
        Amu = A[..., mu]
        s = torch.zeros_like(Amu)
        for nu in range(4):
            if nu == mu:
                continue
            Anu = A[..., nu]
            # staple through x + nu: A_nu(x) + A_mu(x+nu) - A_nu(x+mu)
            up = Anu + torch.roll(Amu, -1, dims=nu) - torch.roll(Anu, -1, dims=mu)
            # staple through x - nu: -A_nu(x-nu) + A_mu(x-nu) + A_nu(x-nu+mu)
            Anu_m = torch.roll(Anu, 1, dims=nu)
            dn = -Anu_m + torch.roll(Amu, 1, dims=nu) + torch.roll(Anu_m, -1, dims=mu)
            s = s + torch.sin(up - Amu) + torch.sin(dn - Amu)
        new[..., mu] = Amu + rho * s
    return new


def gauge_field(L, seed: int, sigma_h: float = 0.3, sigma_a: float = 0.2,
                stout_steps: int = 0, rho: float = 0.1, device: str | None = None,
                u1_stout_steps: int = 0):
    """Return (U, A) on the physical lattice L=(L0,L1,L2,L3) as NumPy arrays.

    The random draws come from PCG64(seed) on the host; the exponentials and the
    smearing run in torch on `device` (CUDA when available unless given).
    u1_stout_steps > 0 smears the U(1) angles as well (same rho).
    """
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    rng = _rng(seed)
    H = random_hermitian(rng, V * 4, sigma_h)
    A = rng.normal(0.0, sigma_a, size=(V, 4))
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    Ht = torch.from_numpy(H).to(device)
    U = _expm_i(Ht).reshape(*L, 4, 3, 3)
    del Ht
    for _ in range(int(stout_steps)):
        U = _stout_step(U, L, rho)
    U = U.reshape(V, 4, 3, 3).cpu().numpy()
    if u1_stout_steps:
        A = u1_stout(A, L, u1_stout_steps, rho, device)
    return np.ascontiguousarray(U), np.ascontiguousarray(A)


def u1_stout(A: np.ndarray, L, steps: int, rho: float = 0.1, device: str | None = None) -> np.ndarray:
    """The U(1) angles A [V][4] on the physical lattice L after `steps` abelian
    stout steps with parameter rho (periodic identification)."""
    L = tuple(int(v) for v in L)
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    At = torch.from_numpy(np.asarray(A, dtype=np.float64)).to(device).reshape(*L, 4)
    for _ in range(int(steps)):
        At = _u1_stout_step(At, rho)
    return np.ascontiguousarray(At.reshape(-1, 4).cpu().numpy())


def unit_gauge_field(L):
    """Free field: U = 1, A = 0."""
    V = int(np.prod(L))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for i in range(3):
        U[:, :, i, i] = 1.0
    return U, np.zeros((V, 4))


def spinor(V: int, seed: int, nrhs: int = 0) -> np.ndarray:
    """Gaussian complex spinor field(s): complex128 [V][4][3] or [nrhs][V][4][3]."""
    rng = _rng(seed)
    shape = (V, 4, 3) if nrhs == 0 else (nrhs, V, 4, 3)
    re = rng.normal(0.0, 1.0, size=shape)
    im = rng.normal(0.0, 1.0, size=shape)
    return re + 1j * im


def plaquette(U: np.ndarray, L) -> float:
    """Average Re tr(U_p)/3 over all plaquettes, periodic physical lattice
    (a workload statistic reported beside the smeared fields)."""
    Ut = torch.from_numpy(U).reshape(*L, 4, 3, 3)
    dag = lambda m: m.conj().transpose(-1, -2)
    s, n = 0.0, 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = (Ut[..., mu, :, :] @ torch.roll(Ut[..., nu, :, :], -1, dims=mu)
                 @ dag(torch.roll(Ut[..., mu, :, :], -1, dims=nu)) @ dag(Ut[..., nu, :, :]))
            s += torch.diagonal(P, dim1=-2, dim2=-1).sum(-1).real.mean().item() / 3.0
            n += 1
    return s / n
