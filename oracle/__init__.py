"""Plain FP64 CPU oracle for the MGM method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package. It shares no code with the CUDA library (``paper_2204_06154_gb300``); the only common
module is the seeded input generator ``paper_2204_06154_gb300.inputs``, which holds none of the
method's arithmetic.

The arithmetic lives in ``mgm_oracle.c`` (built by ``oracle.build.build_oracle``); this module
binds it with ctypes and strings the steps together in the order of the paper's Algorithm 2
(preprocessing) and Algorithm 3 (V-cycle), plus right-preconditioned flexible GMRES (Sec. 4.6).

Parity status of every function is pinned by ``tests/test_oracle_*.py``; see the module
docstrings there for what each pin is.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
i64 = C.c_int64


class OracleError(RuntimeError):
    def __init__(self, what, status, row=-1):
        super().__init__(f"oracle {what} failed with status {status} (row {row})")
        self.status = status
        self.row = row


def lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "liboracle.so")
        if not os.path.exists(path):
            from .build import build_oracle
            build_oracle()
        L = C.CDLL(path)
        L.or_knn.argtypes = [f64p, i64, f64p, i64, C.c_int, C.c_int, i32p, C.c_void_p]
        L.or_phs_weights.argtypes = [f64p, f64p, i64, i32p, C.c_int, C.c_int, C.c_int, f64p]
        L.or_phs_weights_rows.argtypes = [f64p, f64p, i64, i32p, C.c_int, C.c_int, C.c_int, i32p, i64, f64p]
        L.or_gfd_weights.argtypes = [f64p, f64p, i64, i32p, C.c_int, C.c_int, C.c_double, f64p]
        L.or_assemble.argtypes = [i64, C.c_int, i32p, f64p, C.c_double, C.c_int, i32p, i32p, f64p]
        L.or_rcm.argtypes = [i64, i32p, i32p, i32p]
        L.or_color.argtypes = [i64, i32p, i32p, C.c_uint64, i32p, C.POINTER(C.c_int32)]
        L.or_priority.argtypes = [C.c_uint64, C.c_uint64]
        L.or_priority.restype = C.c_uint64
        L.or_wse.argtypes = [f64p, i64, i64, C.c_int, i32p, f64p]
        L.or_interp.argtypes = [f64p, i64, f64p, i64, C.c_int, i32p, i32p, f64p]
        L.or_transpose.argtypes = [i64, i64, i32p, i32p, f64p, i32p, i32p, f64p]
        L.or_spgemm.argtypes = [i64, i64, i32p, i32p, f64p, i32p, i32p, f64p, i32p, C.c_void_p, C.c_void_p]
        L.or_lu_factor.argtypes = [f64p, i64, i32p]
        L.or_lu_solve.argtypes = [f64p, i64, i32p, f64p]
        L.or_tangent_basis.argtypes = [f64p, f64p, f64p]
        L.or_last_bad_row.restype = C.c_int64
        L.or_vcycle.argtypes = [C.c_void_p, C.c_int, f64p, i32p, C.c_void_p, C.c_int, C.c_int, f64p, f64p]
        L.or_mgcycle.argtypes = [C.c_void_p, C.c_int, f64p, i32p, C.c_void_p, C.c_int, C.c_int, C.c_int, f64p, f64p]
        L.or_fgmres.argtypes = [i64, i32p, i32p, f64p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int, C.c_int, C.c_int, f64p, f64p, C.c_int, C.c_int, C.c_double,
                                C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_fgmres_cycle.argtypes = L.or_fgmres.argtypes
        L.or_vcycle_bordered.argtypes = [C.c_void_p, C.c_int, C.c_void_p, f64p, i32p, C.c_void_p, C.c_int, C.c_int,
                                         f64p, C.c_double, f64p, C.POINTER(C.c_double)]
        L.or_fgmres_bordered.argtypes = [i64, i32p, i32p, f64p, C.c_void_p, C.c_int, C.c_void_p, f64p, i32p, C.c_void_p,
                                         C.c_int, C.c_int, C.c_int, f64p, f64p, C.c_int, C.c_int, C.c_double,
                                         C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_phs_grad_weights.argtypes = [f64p, f64p, i64, i32p, C.c_int, C.c_int, C.c_int, f64p, f64p]
        L.or_surface_grad.argtypes = [f64p, i64, i32p, C.c_int, f64p, f64p, f64p, f64p]
        L.or_surface_div.argtypes = [f64p, i64, i32p, C.c_int, f64p, f64p, f64p, f64p]
        L.or_bicgstab.argtypes = [i64, i32p, i32p, f64p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_int, C.c_int, f64p, f64p, C.c_int, C.c_double,
                                  C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_mgm_solve.argtypes = [i64, i32p, i32p, f64p, C.c_void_p, C.c_int, f64p, i32p, C.c_void_p,
                                   C.c_int, C.c_int, f64p, f64p, C.c_int, C.c_double,
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.or_mlp_features.argtypes = [i64, C.c_int, i32p, f64p, f64p, f64p, f64p, f64p, f64p]
        L.or_mlp_forward.argtypes = [i64, C.c_int, f64p, f64p, f64p, f64p, f64p, C.c_void_p, C.c_void_p]
        L.or_mlp_vjp.argtypes = [i64, C.c_int, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p]
        _LIB = L
    return _LIB


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(what, st):
    if st != 0:
        raise OracleError(what, st, lib().or_last_bad_row())


# ----------------------------------------------------------------------------------------------
# Step functions (thin wrappers; the arithmetic is in mgm_oracle.c)
# ----------------------------------------------------------------------------------------------
def knn(data, query, k, self_first=False, return_d2=False):
    """k nearest data points of each query point, ascending (d^2, index) (Sec. 2, Sec. 3)."""
    data = _c(data, np.float64); query = _c(query, np.float64)
    idx = np.empty((query.shape[0], k), np.int32)
    d2 = np.empty((query.shape[0], k), np.float64) if return_d2 else None
    _check("knn", lib().or_knn(data, data.shape[0], query, query.shape[0], k, int(self_first), idx,
                               d2.ctypes.data if d2 is not None else None))
    return (idx, d2) if return_d2 else idx


def tangent_basis(n):
    t1 = np.empty(3); t2 = np.empty(3)
    lib().or_tangent_basis(_c(n, np.float64), t1, t2)
    return t1, t2


def phs_weights(xyz, nrm, idx, k, ell, rows=None):
    """Tangent-plane PHS RBF-FD Laplacian weights, one row per stencil (Sec. 2.2). idx holds one
    stencil per point; with rows given, idx holds the stencils of the centres rows (len(rows) x n)
    and the result their weights."""
    xyz = _c(xyz, np.float64); nrm = _c(nrm, np.float64); idx = _c(idx, np.int32)
    nst = xyz.shape[0] if rows is None else len(rows)
    if idx.ndim != 2 or idx.shape[0] != nst or nrm.shape != xyz.shape:
        raise ValueError("phs_weights: idx must hold one stencil per centre and nrm one normal per point")
    if rows is None:
        w = np.empty(idx.shape, np.float64)
        _check("phs_weights", lib().or_phs_weights(xyz, nrm, xyz.shape[0], idx, idx.shape[1], k, ell, w))
    else:
        rows = _c(rows, np.int32)
        w = np.empty((rows.shape[0], idx.shape[1]), np.float64)
        _check("phs_weights", lib().or_phs_weights_rows(xyz, nrm, xyz.shape[0], idx, idx.shape[1], k, ell, rows,
                                                        rows.shape[0], w))
    return w


def phs_grad_weights(xyz, nrm, idx, k, ell):
    """Tangent-plane RBF-FD weights of d/dx^ and d/dy^ at each centre (Sec. 6.3)."""
    idx = _c(idx, np.int32); N, n = idx.shape
    wx = np.empty((N, n)); wy = np.empty((N, n))
    _check("phs_grad_weights", lib().or_phs_grad_weights(_c(xyz, np.float64), _c(nrm, np.float64), N, idx, n, k, ell,
                                                         wx, wy))
    return wx, wy


def surface_grad(nrm, idx, wx, wy, u):
    idx = _c(idx, np.int32); N, n = idx.shape
    g = np.empty((N, 3))
    _check("surface_grad", lib().or_surface_grad(_c(nrm, np.float64), N, idx, n, _c(wx, np.float64), _c(wy, np.float64),
                                                 _c(u, np.float64), g))
    return g


def surface_div(nrm, idx, wx, wy, eta):
    idx = _c(idx, np.int32); N, n = idx.shape
    d = np.empty(N)
    _check("surface_div", lib().or_surface_div(_c(nrm, np.float64), N, idx, n, _c(wx, np.float64), _c(wy, np.float64),
                                               _c(eta, np.float64), d))
    return d


def gfd_weights(xyz, nrm, idx, ell, alpha):
    """Tangent-plane GFD (weighted least squares) Laplacian weights (Sec. 2.3)."""
    xyz = _c(xyz, np.float64); nrm = _c(nrm, np.float64); idx = _c(idx, np.int32)
    w = np.empty(idx.shape, np.float64)
    _check("gfd_weights", lib().or_gfd_weights(xyz, nrm, xyz.shape[0], idx, idx.shape[1], ell, alpha, w))
    return w


def assemble(idx, w, mu=1.0, poisson=False):
    """L = I - mu D (or L = D) as scipy CSR with ascending columns (Sec. 2)."""
    idx = _c(idx, np.int32); w = _c(w, np.float64)
    N, n = idx.shape
    rp = np.empty(N + 1, np.int32); ci = np.empty(N * n, np.int32); v = np.empty(N * n, np.float64)
    _check("assemble", lib().or_assemble(N, n, idx, w, mu, int(poisson), rp, ci, v))
    return sp.csr_matrix((v, ci, rp), shape=(N, N))


def _csr(A):
    A = sp.csr_matrix(A)
    return _c(A.indptr, np.int32), _c(A.indices, np.int32), _c(A.data, np.float64)


def rcm(A):
    """Reverse Cuthill-McKee ordering perm[new] = old of the symmetrised pattern (Sec. 4.2)."""
    rp, ci, _ = _csr(A)
    N = A.shape[0]
    perm = np.empty(N, np.int32)
    _check("rcm", lib().or_rcm(N, rp, ci, perm))
    return perm


def color(A, seed):
    """Greedy colouring in decreasing SplitMix64 priority (multicolour GS ordering)."""
    rp, ci, _ = _csr(A)
    N = A.shape[0]
    col = np.empty(N, np.int32)
    nc = C.c_int32(0)
    _check("color", lib().or_color(N, rp, ci, seed, col, C.byref(nc)))
    return col, int(nc.value)


def priority(seed, i):
    return int(lib().or_priority(seed, i))


def wse(xyz, NH, mode=1):
    """Weighted sample elimination to NH points (Sec. 4.1); mode 0 sequential, 1 rounds."""
    xyz = _c(xyz, np.float64)
    keep = np.empty(NH, np.int32)
    rmax = np.empty(1)
    _check("wse", lib().or_wse(xyz, xyz.shape[0], NH, mode, keep, rmax))
    return keep, float(rmax[0])


def interp(xf, xc, m=3):
    """PHS (phi = r, constant) interpolation I_H^h, N_f x N_c CSR (Sec. 3)."""
    xf = _c(xf, np.float64); xc = _c(xc, np.float64)
    Nf, Nc = xf.shape[0], xc.shape[0]
    rp = np.empty(Nf + 1, np.int32); ci = np.empty(Nf * m, np.int32); v = np.empty(Nf * m, np.float64)
    _check("interp", lib().or_interp(xf, Nf, xc, Nc, m, rp, ci, v))
    nnz = int(rp[-1])
    return sp.csr_matrix((v[:nnz].copy(), ci[:nnz].copy(), rp), shape=(Nf, Nc))


def transpose(A):
    rp, ci, v = _csr(A)
    nr, nc = A.shape
    trp = np.empty(nc + 1, np.int32); tci = np.empty(len(ci), np.int32); tv = np.empty(len(ci), np.float64)
    _check("transpose", lib().or_transpose(nr, nc, rp, ci, v, trp, tci, tv))
    return sp.csr_matrix((tv, tci, trp), shape=(nc, nr))


def spgemm(A, B):
    """C = A B with per-row accumulation in A's column order (Sec. 4.2, eq. (galerkin))."""
    ap, ac, av = _csr(A); bp, bc, bv = _csr(B)
    nA = A.shape[0]; ncB = B.shape[1]
    cp = np.empty(nA + 1, np.int32)
    L = lib()
    _check("spgemm", L.or_spgemm(nA, ncB, ap, ac, av, bp, bc, bv, cp, None, None))
    nnz = int(cp[-1])
    cc = np.empty(max(nnz, 1), np.int32); cv = np.empty(max(nnz, 1), np.float64)
    _check("spgemm", L.or_spgemm(nA, ncB, ap, ac, av, bp, bc, bv, cp, cc.ctypes.data, cv.ctypes.data))
    return sp.csr_matrix((cv[:nnz], cc[:nnz], cp), shape=(nA, ncB))


def galerkin(L, P, R=None):
    """L_H = R L P with R = P^T (Sec. 4.2, eq. (galerkin)), computed as R (L P)."""
    if R is None:
        R = transpose(P)
    return spgemm(R, spgemm(L, P))


def lu_factor(A):
    a = _c(np.asarray(A.todense() if sp.issparse(A) else A), np.float64).copy()
    n = a.shape[0]
    piv = np.empty(n, np.int32)
    _check("lu_factor", lib().or_lu_factor(a, n, piv))
    return a, piv


def lu_solve(lu, piv, b):
    x = _c(b, np.float64).copy()
    lib().or_lu_solve(lu, lu.shape[0], piv, x)
    return x


def permute(A, perm):
    """B = A[perm][:, perm] (perm[new] = old), columns ascending; values copied exactly."""
    B = sp.csr_matrix(A)[perm][:, perm]
    B.sort_indices()
    return sp.csr_matrix(B)


def num_levels(N1, n_min):
    """p = floor(log(N1/N_min)/log 4) + 1 (Alg. 2, number of levels), evaluated exactly in integers as
    1 + the largest t with N_min * 4**t <= N1 (so N_min <= N_p < 4 N_min)."""
    if N1 < n_min:
        return 1
    t = 0
    while n_min * 4 ** (t + 1) <= N1:
        t += 1
    return t + 1


# ----------------------------------------------------------------------------------------------
# Operator construction (Sec. 2) and hierarchy (Alg. 2)
# ----------------------------------------------------------------------------------------------
def build_operator(xyz, nrm, n, method="rbf", k=1, ell=2, mu=1.0, alpha=4.0, poisson=False):
    idx = knn(xyz, xyz, n, self_first=True)
    if method == "rbf":
        w = phs_weights(xyz, nrm, idx, k, ell)
    elif method == "gfd":
        w = gfd_weights(xyz, nrm, idx, ell, alpha)
    else:
        raise ValueError(method)
    return idx, w, assemble(idx, w, mu, poisson)


class _Level(C.Structure):
    _fields_ = [("n", C.c_int64),
                ("rp", C.c_void_p), ("ci", C.c_void_p), ("v", C.c_void_p),
                ("cptr", C.c_void_p), ("crows", C.c_void_p), ("ncol", C.c_int32),
                ("pp", C.c_void_p), ("pc", C.c_void_p), ("pv", C.c_void_p),
                ("rrp", C.c_void_p), ("rc", C.c_void_p), ("rv", C.c_void_p)]


@dataclass
class Hierarchy:
    X: list = field(default_factory=list)      # level point clouds, in each level's RCM order
    L: list = field(default_factory=list)      # level operators (CSR), RCM order
    P: list = field(default_factory=list)      # P[j]: N_j x N_{j+1} interpolation
    R: list = field(default_factory=list)      # R[j] = P[j]^T
    perm: list = field(default_factory=list)   # perm[j][new] = old index within the level's input order
    keep: list = field(default_factory=list)   # keep[j]: WSE survivors of level j (indices of level j)
    colors: list = field(default_factory=list)
    ncolors: list = field(default_factory=list)
    lu: np.ndarray = None
    piv: np.ndarray = None
    cvec: list = field(default_factory=list)   # bordered (Poisson) hierarchies: border vector per level
    blu: np.ndarray = None                     # LU factors of the bordered coarsest matrix
    bpiv: np.ndarray = None
    smoother: str = "mc"
    nu1: int = 1
    nu2: int = 1
    _keep_alive: list = field(default_factory=list)

    @property
    def p(self):
        return len(self.L)

    def _levels(self):
        arrs = []
        lv = (_Level * self.p)()
        for j in range(self.p):
            A = self.L[j]
            rp, ci, v = _csr(A)
            arrs += [rp, ci, v]
            lv[j].n = A.shape[0]
            lv[j].rp, lv[j].ci, lv[j].v = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
            if self.smoother == "mc" and j < self.p - 1:
                col = self.colors[j]
                order = np.argsort(col, kind="stable").astype(np.int32)
                cptr = np.zeros(self.ncolors[j] + 1, np.int32)
                cptr[1:] = np.cumsum(np.bincount(col, minlength=self.ncolors[j]))
                arrs += [order, cptr]
                lv[j].cptr, lv[j].crows, lv[j].ncol = cptr.ctypes.data, order.ctypes.data, self.ncolors[j]
            else:
                lv[j].cptr, lv[j].crows, lv[j].ncol = None, None, 0
            if j < self.p - 1:
                pp, pc, pv = _csr(self.P[j]); rr, rc, rv = _csr(self.R[j])
                arrs += [pp, pc, pv, rr, rc, rv]
                lv[j].pp, lv[j].pc, lv[j].pv = pp.ctypes.data, pc.ctypes.data, pv.ctypes.data
                lv[j].rrp, lv[j].rc, lv[j].rv = rr.ctypes.data, rc.ctypes.data, rv.ctypes.data
        self._keep_alive = arrs + [lv]
        return lv


def setup(xyz, L1, n_min, m=3, seed=0, smoother="mc", nu1=1, nu2=1, wse_mode=1, bordered=False):
    """MGM preprocessing (Alg. 2), in the paper's order:
    RCM of L_1 and X_1; the number of levels p; for each level: WSE coarsening to
    floor(N_1/4^j) points, interpolation, restriction = transpose, Galerkin product (operand
    order of eq. (galerkin)), RCM of L_{j+1} and the matching reordering of the coarse index of
    the transfers; finally the LU factors of L_p. Colourings for the
    multicolour smoother are computed on the final (RCM-ordered) level operators."""
    H = Hierarchy(smoother=smoother, nu1=nu1, nu2=nu2)
    N1 = L1.shape[0]
    perm1 = rcm(L1)
    H.perm.append(perm1)
    H.X.append(_c(xyz, np.float64)[perm1])
    H.L.append(permute(L1, perm1))
    p = num_levels(N1, n_min)
    for j in range(1, p):
        NH = N1 // 4 ** j
        keep, _ = wse(H.X[j - 1], NH, mode=wse_mode)
        H.keep.append(keep)
        Xc = H.X[j - 1][keep]
        P = interp(H.X[j - 1], Xc, m)
        R = transpose(P)
        Lc = galerkin(H.L[j - 1], P, R)
        perm = rcm(Lc)
        H.perm.append(perm)
        H.X.append(Xc[perm])
        H.L.append(permute(Lc, perm))
        P = sp.csr_matrix(P[:, perm]); P.sort_indices()
        H.P.append(P)
        H.R.append(transpose(P))
    for j in range(p - 1):
        c, nc = color(H.L[j], seed)
        H.colors.append(c); H.ncolors.append(nc)
    H.lu, H.piv = lu_factor(H.L[-1])
    if bordered:
        # eq. (gco_saddle_point): c_0 = 1, c_{j+1} = R_j c_j; coarsest [L_p c_p; c_p^T 0]
        H.cvec.append(np.ones(N1))
        for j in range(p - 1):
            H.cvec.append(np.ascontiguousarray(H.R[j] @ H.cvec[j]))
        np_ = H.L[-1].shape[0]
        B = np.zeros((np_ + 1, np_ + 1))
        B[:np_, :np_] = H.L[-1].toarray()
        B[:np_, np_] = H.cvec[-1]
        B[np_, :np_] = H.cvec[-1]
        H.blu, H.bpiv = lu_factor(B)
    return H


def vcycle(H, f, u=None):
    """One V(nu1, nu2) cycle (Alg. 3) for right-hand side f (caller order); u is the initial
    guess (zero when None). Returns the new u."""
    f = _c(f, np.float64)
    u = np.zeros_like(f) if u is None else _c(u, np.float64).copy()
    if H.p == 1:
        return lu_solve(H.lu, H.piv, f[H.perm[0]])[np.argsort(H.perm[0])]
    lv = H._levels()
    _check("vcycle", lib().or_vcycle(C.addressof(lv), H.p, H.lu, H.piv, H.perm[0].ctypes.data, H.nu1, H.nu2, f, u))
    return u


def mgcycle(H, f, cycle="V", u=None):
    """One multigrid cycle of type "V", "W" or "F" (recursive definitions; see or_mgcycle) for the
    right-hand side f (caller order) from the initial guess u (zero when None)."""
    f = _c(f, np.float64)
    u = np.zeros_like(f) if u is None else _c(u, np.float64).copy()
    lv = H._levels()
    _check("mgcycle", lib().or_mgcycle(C.addressof(lv), H.p, H.lu, H.piv, H.perm[0].ctypes.data, H.nu1, H.nu2,
                                       {"V": 0, "W": 1, "F": 2}[cycle], f, u))
    return u


def fgmres(A, H, f, x0=None, restart=50, maxit=200, tol=1e-10, precond=True, hist=False, cycle="V"):
    """Right-preconditioned FGMRES(restart) with one MGM cycle per iteration (Sec. 4.6; a V-cycle,
    or with cycle="W" / "F" a W- or F-cycle). Returns (x, iterations, true relative residual[, history])."""
    rp, ci, v = _csr(A)
    n = A.shape[0]
    f = _c(f, np.float64)
    x = np.zeros(n) if x0 is None else _c(x0, np.float64).copy()
    it = C.c_int(0); rel = C.c_double(0.0)
    hbuf = np.zeros(maxit + 1)
    if H is not None and H.p > 1:
        lv = H._levels(); lvp = C.addressof(lv); p = H.p
        lu, piv, perm = H.lu.ctypes.data, H.piv.ctypes.data, H.perm[0].ctypes.data
    else:
        lvp, p, lu, piv, perm = None, 0, None, None, None
        if precond:
            raise ValueError("FGMRES with a one-level hierarchy: use a direct solve")
    if cycle == "V":
        st = lib().or_fgmres(n, rp, ci, v, lvp, p, lu, piv, perm, H.nu1 if H else 1, H.nu2 if H else 1,
                             int(precond), f, x, restart, maxit, tol, C.byref(it), C.byref(rel), hbuf.ctypes.data)
    else:
        if not precond or p < 2:
            raise ValueError("W and F cycles need a multilevel preconditioner")
        st = lib().or_fgmres_cycle(n, rp, ci, v, lvp, p, lu, piv, perm, H.nu1, H.nu2, {"W": 1, "F": 2}[cycle], f, x,
                                   restart, maxit, tol, C.byref(it), C.byref(rel), hbuf.ctypes.data)
    if st not in (0, 3):
        _check("fgmres", st)
    out = (x, it.value, rel.value)
    return out + (hbuf[: it.value + 1],) if hist else out


def _cvec_ptrs(H):
    arr = (C.c_void_p * H.p)(*[c.ctypes.data for c in H.cvec])
    return arr


def vcycle_bordered(H, r, s):
    """One bordered V-cycle (Sec. 4.4) from a zero guess: (r, s) -> (e, mu), r in caller order."""
    r = _c(r, np.float64)
    e = np.zeros_like(r); mu = C.c_double(0.0)
    lv = H._levels(); cv = _cvec_ptrs(H)
    _check("vcycle_bordered", lib().or_vcycle_bordered(C.addressof(lv), H.p, C.addressof(cv), H.blu, H.bpiv,
                                                       H.perm[0].ctypes.data, H.nu1, H.nu2, r, float(s), e,
                                                       C.byref(mu)))
    return e, mu.value


def fgmres_bordered(A, H, f, tol=1e-10, restart=50, maxit=200, precond=True, hist=False):
    """FGMRES on the bordered system [A 1; 1^T 0][u; lambda] = [f; 0] (eq. (saddle_point)) with the
    bordered MGM V-cycle as right preconditioner. Returns (u, lambda, iterations, true relative
    residual of the bordered system[, history])."""
    rp, ci, v = _csr(A)
    n = A.shape[0]
    fb = np.zeros(n + 1); fb[:n] = _c(f, np.float64)
    x = np.zeros(n + 1)
    it = C.c_int(0); rel = C.c_double(0.0)
    hbuf = np.zeros(maxit + 1)
    lv = H._levels(); cv = _cvec_ptrs(H)
    st = lib().or_fgmres_bordered(n, rp, ci, v, C.addressof(lv), H.p, C.addressof(cv), H.blu, H.bpiv,
                                  H.perm[0].ctypes.data, H.nu1, H.nu2, int(precond), fb, x, restart, maxit, tol,
                                  C.byref(it), C.byref(rel), hbuf.ctypes.data)
    if st not in (0, 3):
        _check("fgmres_bordered", st)
    out = (x[:n].copy(), float(x[n]), it.value, rel.value)
    return out + (hbuf[: it.value + 1],) if hist else out


def bicgstab(A, H, f, x0=None, maxit=200, tol=1e-10, precond=True, hist=False):
    """Right-preconditioned BiCGSTAB with one MGM V-cycle per preconditioner application
    (Sec. 4.6). Returns (x, preconditioner applications, true relative residual[, history])."""
    rp, ci, v = _csr(A)
    n = A.shape[0]
    f = _c(f, np.float64)
    x = np.zeros(n) if x0 is None else _c(x0, np.float64).copy()
    it = C.c_int(0); rel = C.c_double(0.0)
    hbuf = np.zeros(maxit + 1)
    if H is not None and H.p > 1:
        lv = H._levels(); lvp = C.addressof(lv); p = H.p
        lu, piv, perm = H.lu.ctypes.data, H.piv.ctypes.data, H.perm[0].ctypes.data
    else:
        lvp, p, lu, piv, perm = None, 0, None, None, None
        if precond:
            raise ValueError("BiCGSTAB with a one-level hierarchy: use a direct solve")
    st = lib().or_bicgstab(n, rp, ci, v, lvp, p, lu, piv, perm, H.nu1 if H else 1, H.nu2 if H else 1,
                           int(precond), f, x, maxit, tol, C.byref(it), C.byref(rel), hbuf.ctypes.data)
    if st not in (0, 3):
        _check("bicgstab", st)
    out = (x, it.value, rel.value)
    return out + (hbuf[: it.value + 1],) if hist else out


def mgm_solve(A, H, f, x0=None, maxit=200, tol=1e-10):
    """MGM as a standalone solver: repeated V-cycles (Sec. 5.1)."""
    rp, ci, v = _csr(A)
    n = A.shape[0]
    x = np.zeros(n) if x0 is None else _c(x0, np.float64).copy()
    lv = H._levels()
    it = C.c_int(0); rel = C.c_double(0.0)
    lib().or_mgm_solve(n, rp, ci, v, C.addressof(lv), H.p, H.lu, H.piv, H.perm[0].ctypes.data, H.nu1, H.nu2,
                       _c(f, np.float64), x, maxit, tol, C.byref(it), C.byref(rel))
    return x, it.value, rel.value


# ----------------------------------------------------------------------------------------------
# Learned smoother (an addition to the paper's method; see mgm_oracle.c for the definitions)
# ----------------------------------------------------------------------------------------------
def mlp_features(idx, xyz, nrm, w, r):
    """Per-point features (N x 4n) and residual scales rho (N)."""
    idx = _c(idx, np.int32); N, n = idx.shape
    feat = np.empty((N, 4 * n)); rho = np.empty(N)
    _check("mlp_features", lib().or_mlp_features(N, n, idx, _c(xyz, np.float64), _c(nrm, np.float64),
                                                 _c(w, np.float64), _c(r, np.float64), feat, rho))
    return feat, rho


def mlp_forward(W1, W2, w3, feat):
    feat = _c(feat, np.float64); N, din = feat.shape
    out = np.empty(N)
    _check("mlp_forward", lib().or_mlp_forward(N, din, _c(W1, np.float64), _c(W2, np.float64), _c(w3, np.float64),
                                               feat, out, None, None))
    return out


def mlp_vjp(W1, W2, w3, feat, gout):
    """Gradients of sum_i gout_i * out_i with respect to (W1, W2, w3)."""
    feat = _c(feat, np.float64); N, din = feat.shape
    g1 = np.empty((64, din)); g2 = np.empty((64, 64)); g3 = np.empty(64)
    _check("mlp_vjp", lib().or_mlp_vjp(N, din, _c(W1, np.float64), _c(W2, np.float64), _c(w3, np.float64),
                                       feat, _c(gout, np.float64), g1, g2, g3))
    return g1, g2, g3


def mlp_backward(W1, W2, w3, feat, target):
    """Mean-squared-error loss mean_i (out_i - t_i)^2 and its gradients (through mlp_vjp)."""
    out = mlp_forward(W1, W2, w3, feat)
    e = out - _c(target, np.float64)
    g1, g2, g3 = mlp_vjp(W1, W2, w3, feat, 2.0 * e / len(e))
    return float(np.mean(e * e)), g1, g2, g3


def learned_correction(L, idx, xyz, nrm, w, r, W1, W2, w3):
    """delta_i = rho_i * out_i / l_ii for residual r (caller order)."""
    feat, rho = mlp_features(idx, xyz, nrm, w, r)
    return rho * mlp_forward(W1, W2, w3, feat) / L.diagonal()


def learned_loss(L, idx, xyz, nrm, w, r, W1, W2, w3):
    """Training objective of the learned correction: the residual it leaves, relative,
    J = |r - L delta|^2 / |r|^2, and dJ/d(W1, W2, w3). With s = r - L delta,
    dJ/d out_i = -2 (rho_i / l_ii) (L^T s)_i / |r|^2 (the SpMVs are scipy's)."""
    r = _c(r, np.float64)
    feat, rho = mlp_features(idx, xyz, nrm, w, r)
    sc = rho / L.diagonal()
    d = sc * mlp_forward(W1, W2, w3, feat)
    s = r - L @ d
    rr = float(r @ r)
    gout = -2.0 * sc * (L.T @ s) / rr
    g1, g2, g3 = mlp_vjp(W1, W2, w3, feat, gout)
    return float(s @ s) / rr, g1, g2, g3


# ----------------------------------------------------------------------------------------------
# Heat method for geodesic distance (Sec. 6.3)
# ----------------------------------------------------------------------------------------------
def heat_geodesic(xyz, nrm, source, n=30, ell_lap=2, ell_grad=2, k=1, dt=0.01, steps=3, n_min=250, tol=1e-10):
    """The three steps of Sec. 6.3: backward-Euler heat steps (I - dt D) u^{k+1} = u^k from a unit
    spike at `source`; eta = -grad u / |grad u|; the mean-zero Poisson problem D phi = div eta
    (the bordered system of Sec. 4.4). Returns phi - phi[source] (the distance estimate), and the
    iteration counts. The time step must let the heat reach the whole surface above the solver's
    noise floor (u far away ~ exp(-d / sqrt(dt)) against a relative tolerance tol): dt = 0.01 on
    a unit-size surface; dt = h^2 leaves the far-field gradient direction to round-off."""
    N = len(xyz)
    idx = knn(xyz, xyz, n, self_first=True)
    w = phs_weights(xyz, nrm, idx, k, ell_lap)
    Lh = assemble(idx, w, dt)
    H1 = setup(xyz, Lh, n_min)
    u = np.zeros(N); u[source] = 1.0
    its = []
    for _ in range(steps):
        u, it, rel = fgmres(Lh, H1, u, tol=tol)
        its.append(it)
    wx, wy = phs_grad_weights(xyz, nrm, idx, k, ell_grad)
    g = surface_grad(nrm, idx, wx, wy, u)
    eta = -g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    div = surface_div(nrm, idx, wx, wy, eta)
    D = assemble(idx, w, 1.0, poisson=True)
    H2 = setup(xyz, D, n_min, bordered=True)
    phi, lam, it, rel = fgmres_bordered(D, H2, div, tol=tol)
    its.append(it)
    return phi - phi[source], its


def eigs_smallest(L, nev):
    """Eigenpairs of L of smallest magnitude, by the plain definition: a dense eigen-decomposition
    (small N only). Sec. 6.1 finds the same pairs by Arnoldi on the shifted inverse (shift -1 for
    the operator -D, i.e. L = I - D). Returns (eigenvalues, N x nev eigenvectors), increasing |lambda|."""
    A = L.toarray() if sp.issparse(L) else np.asarray(L)
    lam, V = np.linalg.eig(A)
    o = np.argsort(np.abs(lam), kind="stable")[:nev]
    return lam[o], V[:, o]


# ----------------------------------------------------------------------------------------------
# Reaction-diffusion pattern formation (Sec. 6.2)
# ----------------------------------------------------------------------------------------------
def reaction_terms(model, u, v, prm):
    """Reaction terms (f, g) of u_t = Du Lap u + f, v_t = Dv Lap v + g.
    "gm": Gierer-Meinhardt, eq. (turing): f = A - B u + u^2 / (v (1 + C u^2)), g = u^2 - v,
    prm = (A, B, C). "schnakenberg": f = gamma (a - u + u^2 v), g = gamma (b - u^2 v),
    prm = (gamma, a, b)."""
    if model == "gm":
        A, B, Cc = prm
        return A - B * u + u * u / (v * (1.0 + Cc * u * u)), u * u - v
    gamma, a, b = prm
    return gamma * (a - u + u * u * v), gamma * (b - u * u * v)


def reaction_diffusion(xyz, nrm, model, prm, Du, Dv, dt, steps, u0, v0, scheme="sbdf2", n=30, ell=3, k=1, n_min=250,
                       tol=1e-8):
    """Semi-implicit time stepping of Sec. 6.2: diffusion implicit, reactions explicit, each step
    two screened-Poisson solves (MGM-FGMRES from the previous step's values). scheme "sbdf2"
    (the paper's): (3 w^{n+1} - 4 w^n + w^{n-1}) / (2 dt) = D Lap w^{n+1} + 2 r^n - r^{n-1}, i.e.
    (I - (2/3) dt D Lap) w^{n+1} = (4 w^n - w^{n-1}) / 3 + (2/3) dt (2 r^n - r^{n-1}), its first step
    by IMEX Euler; scheme "euler": (I - dt D Lap) w^{n+1} = w^n + dt r^n. Returns (u, v, iterations
    of every solve)."""
    idx = knn(xyz, xyz, n, self_first=True)
    w = phs_weights(xyz, nrm, idx, k, ell)
    ops = {}

    def op(mu):
        if mu not in ops:
            Lm = assemble(idx, w, mu)
            ops[mu] = (Lm, setup(xyz, Lm, n_min))
        return ops[mu]

    u, v = np.array(u0, np.float64), np.array(v0, np.float64)
    up = vp = None
    its = []
    for step in range(steps):
        f, g = reaction_terms(model, u, v, prm)
        if scheme == "euler" or step == 0:
            ru, rv = u + dt * f, v + dt * g
            cu, cv = dt * Du, dt * Dv
        else:
            fp, gp = reaction_terms(model, up, vp, prm)
            ru = (4.0 * u - up) / 3.0 + (2.0 / 3.0) * dt * (2.0 * f - fp)
            rv = (4.0 * v - vp) / 3.0 + (2.0 / 3.0) * dt * (2.0 * g - gp)
            cu, cv = (2.0 / 3.0) * dt * Du, (2.0 / 3.0) * dt * Dv
        Lu, Hu = op(cu)
        Lv, Hv = op(cv)
        un, itu, _ = fgmres(Lu, Hu, ru, x0=u, tol=tol)
        vn, itv, _ = fgmres(Lv, Hv, rv, x0=v, tol=tol)
        its.append((itu, itv))
        up, vp, u, v = u, v, un, vn
    return u, v, its
