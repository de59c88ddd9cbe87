"""Thin ctypes binding of libqxd (include/qxd.h): argument marshalling only.

Arrays may be NumPy arrays (host memory) or CUDA torch tensors (device memory);
the library itself decides whether to stage them.  Every function raises
QxdError when the C call returns a non-zero status.  There is no fallback: if
libqxd.so has not been built (``paper_1908_11673_gb300.build``) or no CUDA
device is present, loading fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libqxd.so")

FP64, FP32, BF16 = 0, 1, 2
CGNE, FGCR, MSCG = 0, 1, 2
PRECOND_NONE, PRECOND_LEARNED, PRECOND_SAP, PRECOND_DFL = 0, 1, 2, 3
TBC_PERIODIC, TBC_OPEN = 0, 1
LOSS_ERROR, LOSS_RESIDUAL = 0, 1

STATUS = {0: "QXD_OK", 1: "QXD_EARG", 2: "QXD_ENOCONV", 3: "QXD_EBREAKDOWN", 4: "QXD_ENAN",
          5: "QXD_ECUDA", 6: "QXD_ENOMEM", 7: "QXD_ESTATE"}

EXPORTS = ["qxd_create", "qxd_destroy", "qxd_set_links", "qxd_set_clover", "qxd_apply_Dw",
           "qxd_apply_Dhat_eo", "qxd_apply_Dhat_eo_noalloc", "qxd_solve", "qxd_solve_multishift", "qxd_set_precond_weights",
           "qxd_set_sap", "qxd_sap_apply", "qxd_ptc_apply", "qxd_ptc_loss_grad", "qxd_ptc_train", "qxd_ptc_record_pairs",
           "qxd_rat_apply", "qxd_pf_action", "qxd_rw_rat", "qxd_rw_rtm", "qxd_sdet",
           "qxd_dfl_setup", "qxd_dfl_basis", "qxd_dfl_little", "qxd_dfl_apply",
           "qxd_rat_residues", "qxd_rtm_residues", "qxd_block_neighbours",
           "qxd_profile", "qxd_profile_entry", "qxd_last_error", "qxd_volume"]


class QxdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Geom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("cstar", ctypes.c_int), ("theta", ctypes.c_double * 4),
                ("tbc", ctypes.c_int), ("cF", ctypes.c_double)]


class Flavour(ctypes.Structure):
    _fields_ = [("qhat", ctypes.c_int), ("kappa", ctypes.c_double), ("su3csw", ctypes.c_double),
                ("u1csw", ctypes.c_double)]


class Solver(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("tol", ctypes.c_double), ("nmx", ctypes.c_int), ("nkv", ctypes.c_int),
                ("inner", ctypes.c_int), ("inner_tol", ctypes.c_double), ("precond", ctypes.c_int)]


class Rational(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("A", ctypes.c_double), ("nu", ctypes.POINTER(ctypes.c_double)),
                ("mu", ctypes.POINTER(ctypes.c_double))]


def rational(A, nu, mu):
    """qxd_rational for coefficients (A, nu[], mu[]); keeps the arrays alive on the result."""
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    if nu.shape != mu.shape or nu.ndim != 1:
        raise ValueError("nu and mu must be 1-D arrays of the same length")
    r = Rational(len(nu), float(A), nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    r._keep = (nu, mu)
    return r


class DflParams(ctypes.Structure):
    _fields_ = [("Ns", ctypes.c_int), ("ninv", ctypes.c_int), ("ctol", ctypes.c_double), ("cnmx", ctypes.c_int),
                ("cnkv", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("op_applies", ctypes.c_int), ("true_relres", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIBPATH) -> ctypes.CDLL:
    """Load libqxd.so and declare its signatures (raises OSError if absent)."""
    global _lib
    if _lib is not None and path == LIBPATH:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_1908_11673_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "qxd_create": (i, [ctypes.POINTER(Geom), i, ctypes.POINTER(vp)]),
        "qxd_destroy": (None, [vp]),
        "qxd_set_links": (i, [vp, vp, vp, d, vp]),
        "qxd_set_clover": (i, [vp, i, ctypes.POINTER(Flavour), vp]),
        "qxd_apply_Dw": (i, [vp, i, i, vp, vp, i, vp]),
        "qxd_apply_Dhat_eo": (i, [vp, i, i, i, vp, vp, i, vp]),
        "qxd_apply_Dhat_eo_noalloc": (i, [vp, i, i, i, vp, vp, vp]),
        "qxd_solve": (i, [vp, i, ctypes.POINTER(Solver), vp, vp, i, ctypes.POINTER(Info), vp]),
        "qxd_solve_multishift": (i, [vp, i, i, vp, ctypes.POINTER(Solver), vp, vp, ctypes.POINTER(Info), vp]),
        "qxd_set_precond_weights": (i, [vp, i, vp, i, i, i]),
        "qxd_set_sap": (i, [vp, i, i]),
        "qxd_sap_apply": (i, [vp, i, vp, vp, vp]),
        "qxd_ptc_apply": (i, [vp, i, i, vp, i, i, vp, vp, vp]),
        "qxd_ptc_loss_grad": (i, [vp, i, vp, i, i, vp, vp, i, i, ctypes.POINTER(d), vp, vp]),
        "qxd_ptc_train": (i, [vp, i, vp, vp, vp, i, i, vp, vp, i, i, i, d, i, ctypes.POINTER(i), vp, vp]),
        "qxd_ptc_record_pairs": (i, [vp, i, vp, i, i, vp, vp, vp]),
        "qxd_rat_apply": (i, [vp, i, ctypes.POINTER(Rational), i, i, ctypes.POINTER(Solver), vp, vp,
                              ctypes.POINTER(Info), vp]),
        "qxd_pf_action": (i, [vp, i, ctypes.POINTER(Rational), i, i, ctypes.POINTER(Solver), vp,
                              ctypes.POINTER(d), ctypes.POINTER(Info), vp]),
        "qxd_rw_rat": (i, [vp, i, ctypes.POINTER(Rational), i, i, i, ctypes.POINTER(Solver), vp, vp,
                           ctypes.POINTER(d), ctypes.POINTER(Info), vp]),
        "qxd_rw_rtm": (i, [vp, i, ctypes.POINTER(Rational), ctypes.POINTER(Rational), i, i,
                           ctypes.POINTER(Solver), vp, ctypes.POINTER(d), ctypes.POINTER(Info), vp]),
        "qxd_sdet": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(i), vp]),
        "qxd_dfl_setup": (i, [vp, i, ctypes.POINTER(DflParams), vp, vp]),
        "qxd_dfl_basis": (i, [vp, i, i, vp, vp]),
        "qxd_dfl_little": (i, [vp, i, vp, vp, ctypes.POINTER(i), vp]),
        "qxd_dfl_apply": (i, [vp, i, vp, vp, ctypes.POINTER(Info), vp]),
        "qxd_rat_residues": (i, [ctypes.POINTER(Rational), i, i, vp]),
        "qxd_rtm_residues": (i, [ctypes.POINTER(Rational), ctypes.POINTER(Rational), i, i, vp, vp]),
        "qxd_block_neighbours": (i, [ctypes.POINTER(Geom), vp, ctypes.POINTER(i)]),
        "qxd_profile": (i, [vp, i]),
        "qxd_profile_entry": (i, [vp, i, ctypes.c_char_p, i, ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "qxd_last_error": (ctypes.c_char_p, [vp]),
        "qxd_volume": (ctypes.c_longlong, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIBPATH:
        _lib = lib
    return lib


def rat_residues(r, k, l):
    """Partial-fraction residues sigma_j, j = k..l, of the factor P_{k,l} (host code of the library)."""
    lib = load_library()
    out = np.zeros(max(l - k + 1, 1), dtype=np.float64)
    rc = lib.qxd_rat_residues(ctypes.byref(r), int(k), int(l), out.ctypes.data)
    if rc:
        raise QxdError(rc, "rat_residues: bad arguments or coinciding poles")
    return out


def rtm_residues(r_mu, r_t, k, l):
    """Residues (sigma, sigma_t) of Ptilde_{k,l} - 1 (host code of the library)."""
    lib = load_library()
    s1 = np.zeros(max(l - k + 1, 1), dtype=np.float64)
    s2 = np.zeros(max(l - k + 1, 1), dtype=np.float64)
    rc = lib.qxd_rtm_residues(ctypes.byref(r_mu), ctypes.byref(r_t), int(k), int(l), s1.ctypes.data, s2.ctypes.data)
    if rc:
        raise QxdError(rc, "rtm_residues: bad arguments or coinciding poles")
    return s1, s2


def block_neighbours(L, cstar=0, theta=(np.pi, 0.0, 0.0, 0.0)):
    """Block neighbour table [Nb][9] of the 4^4 block grid (host code of the library)."""
    lib = load_library()
    g = Geom((ctypes.c_int * 4)(*[int(x) for x in L]), int(cstar), (ctypes.c_double * 4)(*[float(t) for t in theta]),
             TBC_PERIODIC, 1.0)
    nb = ctypes.c_int()
    rc = lib.qxd_block_neighbours(ctypes.byref(g), None, ctypes.byref(nb))
    if rc:
        raise QxdError(rc, "block_neighbours: invalid geometry or extents not multiples of 8")
    out = np.zeros((nb.value, 9), dtype=np.int32)
    lib.qxd_block_neighbours(ctypes.byref(g), out.ctypes.data, None)
    return out


def _ptr(a):
    """Address of a NumPy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


class Context:
    """One lattice on one GPU (qxd_create ... qxd_destroy)."""

    def __init__(self, L, cstar=0, theta=(0.0, 0.0, 0.0, 0.0), device=0, tbc=TBC_PERIODIC, cF=1.0):
        self.lib = load_library()
        g = Geom()
        g.L[:] = [int(v) for v in L]
        g.cstar = int(cstar)
        g.theta[:] = [float(t) for t in theta]
        g.tbc = int(tbc)
        g.cF = float(cF)
        self._h = ctypes.c_void_p()
        rc = self.lib.qxd_create(ctypes.byref(g), int(device), ctypes.byref(self._h))
        if rc != 0:
            raise QxdError(rc, "qxd_create failed (geometry or device)")
        self.L = tuple(int(v) for v in L)
        self.cstar = int(cstar)
        self.V = int(self.lib.qxd_volume(self._h))
        self.Vh = self.V // 2

    def _check(self, rc):
        if rc != 0:
            raise QxdError(rc, self.lib.qxd_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.lib.qxd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_links(self, U, A, invqel=6.0, stream=None):
        self._check(self.lib.qxd_set_links(self._h, _ptr(U), _ptr(A), float(invqel), _stream(stream)))

    def set_clover(self, fl, qhat, kappa, su3csw, u1csw, stream=None):
        f = Flavour(int(qhat), float(kappa), float(su3csw), float(u1csw))
        self._check(self.lib.qxd_set_clover(self._h, int(fl), ctypes.byref(f), _stream(stream)))

    def apply_Dw(self, fl, prec, inp, out, nrhs=1, stream=None):
        self._check(self.lib.qxd_apply_Dw(self._h, int(fl), int(prec), _ptr(inp), _ptr(out), int(nrhs),
                                          _stream(stream)))

    def apply_Dhat_eo(self, fl, prec, inp, out, dagger=False, nrhs=1, stream=None):
        self._check(self.lib.qxd_apply_Dhat_eo(self._h, int(fl), int(prec), int(bool(dagger)), _ptr(inp),
                                               _ptr(out), int(nrhs), _stream(stream)))

    def apply_Dhat_eo_noalloc(self, fl, prec, inp, out, dagger=False, stream=None):
        """Dhat without any device allocation (device arrays only, V/2 <= 32768)."""
        self._check(self.lib.qxd_apply_Dhat_eo_noalloc(self._h, int(fl), int(prec), int(bool(dagger)), _ptr(inp),
                                                       _ptr(out), _stream(stream)))

    def solve(self, fl, eta, psi, kind=FGCR, tol=1e-10, nmx=20000, nkv=16, inner=FP32, inner_tol=0.0,
              precond=PRECOND_NONE, nrhs=1, stream=None, check=True):
        s = Solver(int(kind), float(tol), int(nmx), int(nkv), int(inner), float(inner_tol), int(precond))
        info = Info()
        rc = self.lib.qxd_solve(self._h, int(fl), ctypes.byref(s), _ptr(eta), _ptr(psi), int(nrhs),
                                ctypes.byref(info), _stream(stream))
        if check:
            self._check(rc)
        return info

    def solve_multishift(self, fl, sigma, phi_e, x_e, tol=1e-10, nmx=20000, inner=FP64, stream=None,
                         check=True):
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
        s = Solver(MSCG, float(tol), int(nmx), 0, int(inner), 0.0, PRECOND_NONE)
        info = Info()
        rc = self.lib.qxd_solve_multishift(self._h, int(fl), len(sig), sig.ctypes.data, ctypes.byref(s),
                                           _ptr(phi_e), _ptr(x_e), ctypes.byref(info), _stream(stream))
        if check:
            self._check(rc)
        return info

    # ---- rational factors, reweighting, small determinant (App. A.2, A.3) -------
    def _msolver(self, tol, nmx, inner):
        return Solver(MSCG, float(tol), int(nmx), 0, int(inner), 0.0, PRECOND_NONE)

    def rat_apply(self, fl, r, k, l, in_e, out_e, tol=1e-10, nmx=20000, inner=FP32, stream=None):
        """out_e = P_{k,l} in_e (r: a qxd.Rational from qxd.rational)."""
        info = Info()
        s = self._msolver(tol, nmx, inner)
        self._check(self.lib.qxd_rat_apply(self._h, int(fl), ctypes.byref(r), int(k), int(l), ctypes.byref(s),
                                           _ptr(in_e), _ptr(out_e), ctypes.byref(info), _stream(stream)))
        return info

    def pf_action(self, fl, r, k, l, phi_e, tol=1e-10, nmx=20000, inner=FP32, stream=None):
        """(phi, P_{k,l} phi); returns (S, info)."""
        info = Info()
        S = ctypes.c_double()
        s = self._msolver(tol, nmx, inner)
        self._check(self.lib.qxd_pf_action(self._h, int(fl), ctypes.byref(r), int(k), int(l), ctypes.byref(s),
                                           _ptr(phi_e), ctypes.byref(S), ctypes.byref(info), _stream(stream)))
        return S.value, info

    def rw_rat(self, fl, r, u, v, nterms, eta_e, tol=1e-10, nmx=20000, inner=FP32, stream=None):
        """((eta, Z^n eta) for n = 1..nterms, exponent, info)."""
        info = Info()
        terms = np.zeros(int(nterms), dtype=np.float64)
        e = ctypes.c_double()
        s = self._msolver(tol, nmx, inner)
        self._check(self.lib.qxd_rw_rat(self._h, int(fl), ctypes.byref(r), int(u), int(v), int(nterms),
                                        ctypes.byref(s), _ptr(eta_e), terms.ctypes.data, ctypes.byref(e),
                                        ctypes.byref(info), _stream(stream)))
        return terms, e.value, info

    def rw_rtm(self, fl, r_mu, r_t, k, l, eta_e, tol=1e-10, nmx=20000, inner=FP32, stream=None):
        """((eta, [Ptilde_{k,l} - 1] eta), info)."""
        info = Info()
        e = ctypes.c_double()
        s = self._msolver(tol, nmx, inner)
        self._check(self.lib.qxd_rw_rtm(self._h, int(fl), ctypes.byref(r_mu), ctypes.byref(r_t), int(k), int(l),
                                        ctypes.byref(s), _ptr(eta_e), ctypes.byref(e), ctypes.byref(info),
                                        _stream(stream)))
        return e.value, info

    def sdet(self, fl, stream=None):
        """(sum over odd sites of log|det D_oo(x)|, number of negative determinants)."""
        ld = ctypes.c_double()
        nn = ctypes.c_int()
        self._check(self.lib.qxd_sdet(self._h, int(fl), ctypes.byref(ld), ctypes.byref(nn), _stream(stream)))
        return ld.value, nn.value

    # ---- inexact deflation (DFL+SAP+GCR) ------------------------------------------
    def dfl_setup(self, fl, seeds, Ns, ninv=2, ctol=1e-2, cnmx=64, cnkv=16, stream=None):
        """Build the deflation subspace of flavour fl from seeds (complex64 [Ns][V][4][3])."""
        p = DflParams(int(Ns), int(ninv), float(ctol), int(cnmx), int(cnkv))
        self._check(self.lib.qxd_dfl_setup(self._h, int(fl), ctypes.byref(p), _ptr(seeds), _stream(stream)))

    def dfl_basis(self, fl, k, out, stream=None):
        self._check(self.lib.qxd_dfl_basis(self._h, int(fl), int(k), _ptr(out), _stream(stream)))

    def dfl_little(self, fl, Ns, stream=None):
        """(A [Nb][9][Ns][Ns] complex64 with A[B][s][l][k] = <phi_k|_B, D phi_l|_{B_s}>, nbr [Nb][9])."""
        nb = ctypes.c_int()
        self._check(self.lib.qxd_dfl_little(self._h, int(fl), None, None, ctypes.byref(nb), _stream(stream)))
        A = np.empty((nb.value, 9, Ns, Ns), dtype=np.complex64)
        nbr = np.empty((nb.value, 9), dtype=np.int32)
        self._check(self.lib.qxd_dfl_little(self._h, int(fl), A.ctypes.data, nbr.ctypes.data, None,
                                            _stream(stream)))
        return A, nbr

    def dfl_apply(self, fl, v, out, stream=None):
        info = Info()
        self._check(self.lib.qxd_dfl_apply(self._h, int(fl), _ptr(v), _ptr(out), ctypes.byref(info), _stream(stream)))
        return info

    # ---- SAP preconditioner ----------------------------------------------------
    def set_sap(self, ncy=5, nmr=5):
        self._check(self.lib.qxd_set_sap(self._h, int(ncy), int(nmr)))

    def sap_apply(self, fl, inp, out, stream=None):
        self._check(self.lib.qxd_sap_apply(self._h, int(fl), _ptr(inp), _ptr(out), _stream(stream)))

    # ---- learned preconditioner ------------------------------------------------
    def ptc_apply(self, fl, W, nlayers, nch, inp, out, stream=None, prec=FP32):
        """out_e = (M in_e)_e; prec FP32 (CUDA cores) or BF16 (tensor-core channel mixing)."""
        self._check(self.lib.qxd_ptc_apply(self._h, int(fl), int(prec), _ptr(W), int(nlayers), int(nch), _ptr(inp),
                                           _ptr(out), _stream(stream)))

    def ptc_loss_grad(self, fl, W, nlayers, nch, r, e, npairs, grad=None, stream=None, kind=LOSS_ERROR):
        """Summed loss over the pairs (kind LOSS_ERROR or LOSS_RESIDUAL) and its gradient."""
        loss = ctypes.c_double()
        self._check(self.lib.qxd_ptc_loss_grad(self._h, int(fl), _ptr(W), int(nlayers), int(nch), _ptr(r), _ptr(e),
                                               int(npairs), int(kind), ctypes.byref(loss), _ptr(grad),
                                               _stream(stream)))
        return loss.value

    def ptc_train(self, fl, W, m, v, nlayers, nch, r, e, npairs, batch, nsteps, lr, t, stream=None, kind=LOSS_ERROR):
        """Adam steps on (W, m, v) in place; t is a one-element int32 array (step counter).
        Returns the per-step mean losses."""
        losses = np.zeros(max(nsteps, 1), dtype=np.float64)
        tc = ctypes.c_int(int(t[0]))
        self._check(self.lib.qxd_ptc_train(self._h, int(fl), _ptr(W), _ptr(m), _ptr(v), int(nlayers), int(nch),
                                           _ptr(r), _ptr(e), int(npairs), int(batch), int(nsteps), float(lr), int(kind),
                                           ctypes.byref(tc), losses.ctypes.data, _stream(stream)))
        t[0] = tc.value
        return losses[:nsteps]

    def ptc_record_pairs(self, fl, b, npairs, stride, r_out, e_out, stream=None):
        self._check(self.lib.qxd_ptc_record_pairs(self._h, int(fl), _ptr(b), int(npairs), int(stride), _ptr(r_out),
                                                  _ptr(e_out), _stream(stream)))

    def profile(self, mode):
        """0 off, 1 count kernel launches, 2 count and time them (resets the counters)."""
        self._check(self.lib.qxd_profile(self._h, int(mode)))

    def profile_entries(self):
        """[{name, launches, ms, bytes}] for every kernel class launched since profile()."""
        out = []
        buf = ctypes.create_string_buffer(64)
        n, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        i = 0
        while self.lib.qxd_profile_entry(self._h, i, buf, 64, ctypes.byref(n), ctypes.byref(ms),
                                         ctypes.byref(by)) == 0:
            out.append({"name": buf.value.decode(), "launches": n.value, "ms": ms.value, "bytes": by.value})
            i += 1
        return out

    def set_precond_weights(self, fl, W, nlayers, nch, prec=BF16):
        """Network weights of the learned preconditioner and the precision of its
        channel mixing inside FGCR (BF16: tensor cores; FP32: CUDA cores)."""
        self._check(self.lib.qxd_set_precond_weights(self._h, int(fl), _ptr(W), int(nlayers), int(nch), int(prec)))
