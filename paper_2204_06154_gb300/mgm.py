"""Thin ctypes binding of libmgm (include/mgm.h): argument marshalling only.

Every array is a CUDA torch tensor (device memory and the current stream come from PyTorch); all
computation happens in the library's sm_103a kernels. If libmgm.so is missing the import-time
loader raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libmgm.so")
_lib = None

MGM_RBF_FD, MGM_GFD = 0, 1
MGM_F64, MGM_F32 = 0, 1
MGM_KRYLOV_FGMRES, MGM_KRYLOV_NONE, MGM_KRYLOV_BICGSTAB = 0, 1, 2
_KRYLOV = {"fgmres": MGM_KRYLOV_FGMRES, "none": MGM_KRYLOV_NONE, "bicgstab": MGM_KRYLOV_BICGSTAB, "fgmres_graph": 3}

STATUS = {0: "MGM_OK", 1: "MGM_ERR_INVALID_ARG", 2: "MGM_ERR_SINGULAR_STENCIL", 3: "MGM_ERR_NOT_CONVERGED",
          4: "MGM_ERR_BREAKDOWN", 5: "MGM_ERR_TIMEOUT", 6: "MGM_ERR_CUDA", 7: "MGM_ERR_OOM", 8: "MGM_ERR_UNSUPPORTED"}


class MGMError(RuntimeError):
    def __init__(self, status, message, row=-1):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.row = row


class StencilParams(C.Structure):
    _fields_ = [("method", C.c_int), ("k", C.c_int), ("ell", C.c_int), ("n", C.c_int), ("alpha", C.c_double),
                ("mu", C.c_double), ("poisson", C.c_int), ("weights", C.c_int)]


class Params(C.Structure):
    _fields_ = [("n_min", C.c_int64), ("m", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64), ("persistent_sweeps", C.c_int), ("constraint", C.c_int), ("smoother", C.c_int),
                ("cycle", C.c_int), ("transfer_bf16", C.c_int)]


class SolveParams(C.Structure):
    _fields_ = [("krylov", C.c_int), ("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_len", C.c_int), ("solve_ms", C.c_float), ("multiplier", C.c_double)]


class HierStats(C.Structure):
    _fields_ = [("p", C.c_int), ("precision", C.c_int), ("n", C.c_int64 * 16), ("nnz", C.c_int64 * 16),
                ("ncolors", C.c_int32 * 16), ("device_bytes", C.c_int64)]


EXPORTS = ["mgm_knn", "mgm_knn_noalloc", "mgm_stencil_weights", "mgm_assemble", "mgm_build_stencils", "mgm_coarsen", "mgm_interp",
           "mgm_transpose", "mgm_spgemm", "mgm_rcm", "mgm_color", "mgm_setup", "mgm_vcycle", "mgm_solve", "mgm_solve_multi",
           "mgm_solve_batched",
           "mgm_hierarchy_stats_get", "mgm_hierarchy_level", "mgm_hierarchy_pnnz", "mgm_profile",
           "mgm_kernel_launches", "mgm_check_bounded_wait", "mgm_destroy", "mgm_release_cached_memory", "mgm_status_string", "mgm_last_error_message",
           "mgm_last_error_row", "mgm_last_weights_fp64_rows",
           "mgm_mlp_size", "mgm_mlp_create", "mgm_mlp_destroy", "mgm_mlp_get", "mgm_mlp_set", "mgm_mlp_forward",
           "mgm_mlp_vjp", "mgm_learned_attach", "mgm_learned_features", "mgm_learned_cycle_residual", "mgm_learned_loss",
           "mgm_learned_train_step", "mgm_learned_enable", "mgm_learned_correction", "mgm_learned_info",
           "mgm_gradient_weights", "mgm_surface_gradient", "mgm_surface_divergence", "mgm_eigs", "mgm_reaction_rhs",
           "mgm_sweep_config_set", "mgm_sweep_config_get", "mgm_autotune", "mgm_profile_level", "mgm_reaction_steps",
           "mgm_probe_fp64_fma", "mgm_probe_launch_chain", "mgm_vcycle_floor", "mgm_level_smoothing_bytes", "mgm_tail_info"]


_SCHEDULES = ["launch", "stream", "resident", "colour"]


class SweepConfig(C.Structure):
    _fields_ = [("kind", C.c_int), ("blocks", C.c_int), ("lanes", C.c_int), ("stages", C.c_int), ("ms", C.c_float)]


class ProfileInfo(C.Structure):
    _fields_ = [("vcycle_ms", C.c_float), ("vcycle_bytes", C.c_int64), ("vcycle_kernels", C.c_int64),
                ("sweep_ms", C.c_float), ("sweep_bytes", C.c_int64), ("sweep_launches", C.c_int32),
                ("spmv_ms", C.c_float), ("spmv_bytes", C.c_int64),
                ("learned_vcycle_ms", C.c_float), ("learned_ms", C.c_float), ("learned_bytes", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError(f"{_LIBPATH} is missing: build it with paper_2204_06154_gb300.build.build()")
        L = C.CDLL(_LIBPATH)
        P, I64, I = C.c_void_p, C.c_int64, C.c_int
        L.mgm_knn.argtypes = [P, I64, P, I64, I, I, P, P]
        L.mgm_knn_noalloc.argtypes = [P, I64, P, I64, I, I, P, P]
        L.mgm_stencil_weights.argtypes = [P, P, I64, P, C.POINTER(StencilParams), P, P]
        L.mgm_assemble.argtypes = [I64, I, P, P, C.c_double, I, P, P, P, P]
        L.mgm_build_stencils.argtypes = [P, P, I64, C.POINTER(StencilParams), P, P, P, P, P, P]
        L.mgm_coarsen.argtypes = [P, I64, I64, C.c_uint64, P, P]
        L.mgm_interp.argtypes = [P, I64, P, I64, I, P, P, P, C.POINTER(C.c_int64), P]
        L.mgm_transpose.argtypes = [I64, I64, P, P, P, P, P, P, P]
        L.mgm_spgemm.argtypes = [I64, I64, I64, P, P, P, P, P, P, P, P, P, C.POINTER(C.c_int64), P]
        L.mgm_rcm.argtypes = [I64, P, P, P, P]
        L.mgm_color.argtypes = [I64, P, P, C.c_uint64, P, C.POINTER(C.c_int32), P]
        L.mgm_setup.argtypes = [P, I64, P, P, P, C.POINTER(Params), C.POINTER(P), P]
        L.mgm_vcycle.argtypes = [P, P, P, I, P]
        L.mgm_solve.argtypes = [P, P, P, C.POINTER(SolveParams), C.POINTER(SolveInfo), P]
        L.mgm_solve_multi.argtypes = [P, I, P, P, C.POINTER(SolveParams), C.POINTER(SolveInfo), P]
        L.mgm_solve_batched.argtypes = [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), I, C.POINTER(SolveParams),
                                        C.POINTER(SolveInfo), C.POINTER(C.c_int), P]
        L.mgm_hierarchy_stats_get.argtypes = [P, C.POINTER(HierStats)]
        L.mgm_hierarchy_level.argtypes = [P, I] + [P] * 10 + [P]
        L.mgm_hierarchy_pnnz.argtypes = [P, I, C.POINTER(C.c_int64)]
        L.mgm_profile.argtypes = [P, I, C.POINTER(ProfileInfo), P]
        L.mgm_sweep_config_set.argtypes = [P, I, C.POINTER(SweepConfig), P]
        L.mgm_sweep_config_get.argtypes = [P, I, C.POINTER(SweepConfig)]
        L.mgm_autotune.argtypes = [P, I, I, P]
        L.mgm_profile_level.argtypes = [P, I, I, C.POINTER(C.c_float), P]
        L.mgm_probe_fp64_fma.argtypes = [I, C.POINTER(C.c_double), P]
        L.mgm_probe_launch_chain.argtypes = [I, I, I, I, I, C.POINTER(C.c_double), P]
        L.mgm_vcycle_floor.argtypes = [P, C.c_double, C.c_double] + [C.POINTER(C.c_double)] * 3
        L.mgm_level_smoothing_bytes.argtypes = [P, I, C.POINTER(C.c_int64)]
        L.mgm_tail_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.mgm_check_bounded_wait.argtypes = [I, I64, C.POINTER(C.c_int), P]
        L.mgm_kernel_launches.argtypes = []
        L.mgm_kernel_launches.restype = C.c_int64
        L.mgm_destroy.argtypes = [P]
        L.mgm_destroy.restype = None
        L.mgm_release_cached_memory.argtypes = []
        L.mgm_release_cached_memory.restype = None
        L.mgm_gradient_weights.argtypes = [P, P, I64, P, C.POINTER(StencilParams), P, P, P]
        L.mgm_surface_gradient.argtypes = [P, I64, P, I, P, P, P, P, I, P]
        L.mgm_surface_divergence.argtypes = [P, I64, P, I, P, P, P, P, P]
        L.mgm_mlp_size.argtypes = [I]
        L.mgm_mlp_size.restype = C.c_int64
        L.mgm_mlp_create.argtypes = [I, C.c_uint64, C.POINTER(P)]
        L.mgm_mlp_destroy.argtypes = [P]
        L.mgm_mlp_destroy.restype = None
        L.mgm_mlp_get.argtypes = [P, P]
        L.mgm_mlp_set.argtypes = [P, P]
        L.mgm_mlp_forward.argtypes = [P, P, I64, P, P]
        L.mgm_mlp_vjp.argtypes = [P, P, P, I64, P, P]
        L.mgm_learned_attach.argtypes = [P, P, P, P, P, I, P]
        L.mgm_learned_features.argtypes = [P, P, P, P, P]
        L.mgm_learned_cycle_residual.argtypes = [P, P, P, P]
        L.mgm_learned_loss.argtypes = [P, P, P, C.POINTER(C.c_double), P, P]
        L.mgm_learned_train_step.argtypes = [P, P, P, C.c_float, C.POINTER(C.c_double), P]
        L.mgm_learned_enable.argtypes = [P, P, P]
        L.mgm_learned_correction.argtypes = [P, P, P, P]
        L.mgm_learned_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int64)]
        L.mgm_eigs.argtypes = [P, I, I, I, I, C.c_double, C.POINTER(SolveParams), C.c_uint64, P, P, P, P,
                               C.POINTER(C.c_int), C.POINTER(C.c_int), P]
        L.mgm_reaction_rhs.argtypes = [I, I, I64, P, P, P, P, C.POINTER(C.c_double), C.c_double, P, P, P]
        L.mgm_reaction_steps.argtypes = [P, P, I, C.POINTER(C.c_double), C.c_double, P, P, I, C.POINTER(SolveParams),
                                         C.POINTER(C.c_int), P]
        L.mgm_status_string.restype = C.c_char_p
        L.mgm_last_error_message.restype = C.c_char_p
        L.mgm_last_error_row.restype = C.c_int64
        L.mgm_last_weights_fp64_rows.argtypes = []
        L.mgm_last_weights_fp64_rows.restype = C.c_int64
        for name in EXPORTS:
            if name not in ("mgm_destroy", "mgm_release_cached_memory", "mgm_status_string", "mgm_last_error_message",
                            "mgm_last_error_row", "mgm_last_weights_fp64_rows",
                            "mgm_kernel_launches", "mgm_mlp_size", "mgm_mlp_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        L = lib()
        raise MGMError(st, L.mgm_last_error_message().decode(), int(L.mgm_last_error_row()))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.contiguous()


# ----------------------------------------------------------------------------------------------
def knn(data, query, k, self_first=False):
    data = _dev(data, torch.float64, "data")
    query = data if self_first else _dev(query, torch.float64, "query")
    out = torch.empty((query.shape[0], k), dtype=torch.int32, device=data.device)
    _check(lib().mgm_knn(_p(data), data.shape[0], _p(query), query.shape[0], k, int(self_first), _p(out), _stream()))
    return out


def knn_noalloc(data, query, k, self_first=False, out=None):
    """mgm_knn_noalloc: same result as knn(), using the library's static device scratch instead of
    allocating (see include/mgm.h for its size limit and the no-overlap rule)."""
    data = _dev(data, torch.float64, "data")
    query = data if self_first else _dev(query, torch.float64, "query")
    if out is None:
        out = torch.empty((query.shape[0], k), dtype=torch.int32, device=data.device)
    elif (not isinstance(out, torch.Tensor) or out.dtype != torch.int32 or out.device != data.device
          or not out.is_contiguous() or tuple(out.shape) != (query.shape[0], k)):
        # the library writes nq * k int32 values through this pointer
        raise ValueError(f"out must be a contiguous int32 tensor of shape ({query.shape[0]}, {k}) on {data.device}")
    _check(lib().mgm_knn_noalloc(_p(data), data.shape[0], _p(query), query.shape[0], k, int(self_first), _p(out),
                                 _stream()))
    return out


_WEIGHTS = {"f64": 0, "mixed": 1}


def _sp(n, method="rbf", k=1, ell=2, mu=1.0, alpha=4.0, poisson=False, weights="f64"):
    if weights not in _WEIGHTS:
        raise ValueError(f"weights must be one of {sorted(_WEIGHTS)}")
    return StencilParams(MGM_RBF_FD if method == "rbf" else MGM_GFD, k, ell, n, alpha, mu, int(poisson),
                         _WEIGHTS[weights])


def last_weights_fp64_rows():
    """Stencils that the last weights call with weights="mixed" solved again in FP64."""
    return int(lib().mgm_last_weights_fp64_rows())


def release_cached_memory():
    """mgm_release_cached_memory: hand the library's cached device memory back to the device."""
    lib().mgm_release_cached_memory()


def stencil_weights(xyz, nrm, idx, method="rbf", k=1, ell=2, alpha=4.0, weights="f64"):
    """weights="f64": FP64 elimination; "mixed": FP32 LU with FP64 iterative refinement (PHS only)."""
    xyz = _dev(xyz, torch.float64, "xyz"); nrm = _dev(nrm, torch.float64, "nrm"); idx = _dev(idx, torch.int32, "idx")
    sp = _sp(idx.shape[1], method, k, ell, 1.0, alpha, weights=weights)
    w = torch.empty(idx.shape, dtype=torch.float64, device=xyz.device)
    _check(lib().mgm_stencil_weights(_p(xyz), _p(nrm), xyz.shape[0], _p(idx), C.byref(sp), _p(w), _stream()))
    return w


_RD_MODEL = {"gm": 0, "schnakenberg": 1}
_RD_SCHEME = {"euler": 1, "sbdf2": 2}


def reaction_rhs(model, scheme, u, v, prm, dt, u_prev=None, v_prev=None, out=None):
    """Right-hand sides of one semi-implicit reaction-diffusion step (see mgm_reaction_rhs)."""
    u = _dev(u, torch.float64, "u"); v = _dev(v, torch.float64, "v")
    ru, rv = out if out is not None else (torch.empty_like(u), torch.empty_like(v))
    p3 = (C.c_double * 3)(*[float(t) for t in prm])
    _check(lib().mgm_reaction_rhs(_RD_MODEL[model], _RD_SCHEME[scheme], u.numel(), _p(u), _p(v),
                                  _p(u_prev) if u_prev is not None else None, _p(v_prev) if v_prev is not None else None,
                                  p3, float(dt), _p(ru), _p(rv), _stream()))
    return ru, rv


def probe_fp64_fma(reps=20):
    """The device's FP64 multiply-add rate in GFLOP/s (mgm_probe_fp64_fma)."""
    g = C.c_double(0.0)
    _check(lib().mgm_probe_fp64_fma(reps, C.byref(g), _stream()))
    return g.value


def probe_launch_chain(blocks, threads=256, launches=256, pdl=True, reps=10):
    """Microseconds between consecutive dependent launches of `blocks` x `threads` threads
    (mgm_probe_launch_chain)."""
    us = C.c_double(0.0)
    _check(lib().mgm_probe_launch_chain(blocks, threads, launches, 1 if pdl else 0, reps, C.byref(us), _stream()))
    return us.value


def reaction_steps(Hu, Hv, model, prm, dt, u, v, steps, tol=1e-8, restart=50, maxit=200):
    """IMEX Euler steps on the device, each one graph launch (see mgm_reaction_steps); u and v (CUDA
    float64, caller order) are advanced in place. Returns the (u, v) iteration counts per step."""
    u = _dev(u, torch.float64, "u"); v = _dev(v, torch.float64, "v")
    p3 = (C.c_double * 3)(*[float(t) for t in prm])
    sp = SolveParams(MGM_KRYLOV_FGMRES, restart, maxit, tol)
    its = (C.c_int * (2 * max(steps, 1)))()
    _check(lib().mgm_reaction_steps(Hu._h, Hv._h, _RD_MODEL[model], p3, float(dt), _p(u), _p(v), steps, C.byref(sp),
                                    its, _stream()))
    return [(its[2 * t], its[2 * t + 1]) for t in range(steps)]


def gradient_weights(xyz, nrm, idx, k=1, ell=2):
    """Tangent-plane RBF-FD weights of d/dx^ and d/dy^ (Sec. 6.3)."""
    xyz = _dev(xyz, torch.float64, "xyz"); nrm = _dev(nrm, torch.float64, "nrm"); idx = _dev(idx, torch.int32, "idx")
    sp = _sp(idx.shape[1], "rbf", k, ell, 1.0, 4.0)
    wx = torch.empty(idx.shape, dtype=torch.float64, device=xyz.device)
    wy = torch.empty_like(wx)
    _check(lib().mgm_gradient_weights(_p(xyz), _p(nrm), xyz.shape[0], _p(idx), C.byref(sp), _p(wx), _p(wy), _stream()))
    return wx, wy


def surface_gradient(nrm, idx, wx, wy, u, normalize=False):
    nrm = _dev(nrm, torch.float64, "nrm"); idx = _dev(idx, torch.int32, "idx")
    wx = _dev(wx, torch.float64, "wx"); wy = _dev(wy, torch.float64, "wy"); u = _dev(u, torch.float64, "u")
    g = torch.empty((idx.shape[0], 3), dtype=torch.float64, device=u.device)
    _check(lib().mgm_surface_gradient(_p(nrm), idx.shape[0], _p(idx), idx.shape[1], _p(wx), _p(wy), _p(u), _p(g),
                                      int(normalize), _stream()))
    return g


def surface_divergence(nrm, idx, wx, wy, eta):
    nrm = _dev(nrm, torch.float64, "nrm"); idx = _dev(idx, torch.int32, "idx")
    wx = _dev(wx, torch.float64, "wx"); wy = _dev(wy, torch.float64, "wy"); eta = _dev(eta, torch.float64, "eta")
    d = torch.empty(idx.shape[0], dtype=torch.float64, device=eta.device)
    _check(lib().mgm_surface_divergence(_p(nrm), idx.shape[0], _p(idx), idx.shape[1], _p(wx), _p(wy), _p(eta), _p(d),
                                        _stream()))
    return d


def assemble(idx, w, mu=1.0, poisson=False):
    idx = _dev(idx, torch.int32, "idx"); w = _dev(w, torch.float64, "w")
    N, n = idx.shape
    rp = torch.empty(N + 1, dtype=torch.int32, device=idx.device)
    ci = torch.empty(N * n, dtype=torch.int32, device=idx.device)
    v = torch.empty(N * n, dtype=torch.float64, device=idx.device)
    _check(lib().mgm_assemble(N, n, _p(idx), _p(w), mu, int(poisson), _p(rp), _p(ci), _p(v), _stream()))
    return rp, ci, v


def build_stencils(xyz, nrm, n, method="rbf", k=1, ell=2, mu=1.0, alpha=4.0, poisson=False, keep_weights=True,
                   weights="f64"):
    xyz = _dev(xyz, torch.float64, "xyz"); nrm = _dev(nrm, torch.float64, "nrm")
    N = xyz.shape[0]
    dev = xyz.device
    sp = _sp(n, method, k, ell, mu, alpha, poisson, weights)
    idx = torch.empty((N, n), dtype=torch.int32, device=dev) if keep_weights else None
    w = torch.empty((N, n), dtype=torch.float64, device=dev) if keep_weights else None
    rp = torch.empty(N + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(N * n, dtype=torch.int32, device=dev)
    v = torch.empty(N * n, dtype=torch.float64, device=dev)
    _check(lib().mgm_build_stencils(_p(xyz), _p(nrm), N, C.byref(sp), _p(idx), _p(w), _p(rp), _p(ci), _p(v), _stream()))
    return idx, w, rp, ci, v


def coarsen(xyz, NH):
    xyz = _dev(xyz, torch.float64, "xyz")
    keep = torch.empty(NH, dtype=torch.int32, device=xyz.device)
    _check(lib().mgm_coarsen(_p(xyz), xyz.shape[0], NH, 0, _p(keep), _stream()))
    return keep


def interp(xf, xc, m=3):
    xf = _dev(xf, torch.float64, "xf"); xc = _dev(xc, torch.float64, "xc")
    Nf = xf.shape[0]
    rp = torch.empty(Nf + 1, dtype=torch.int32, device=xf.device)
    ci = torch.empty(Nf * m, dtype=torch.int32, device=xf.device)
    v = torch.empty(Nf * m, dtype=torch.float64, device=xf.device)
    nnz = C.c_int64(0)
    _check(lib().mgm_interp(_p(xf), Nf, _p(xc), xc.shape[0], m, _p(rp), _p(ci), _p(v), C.byref(nnz), _stream()))
    return rp, ci[: nnz.value], v[: nnz.value]


def transpose(nrows, ncols, rp, ci, v):
    nnz = ci.numel()
    trp = torch.empty(ncols + 1, dtype=torch.int32, device=rp.device)
    tci = torch.empty(max(nnz, 1), dtype=torch.int32, device=rp.device)
    tv = torch.empty(max(nnz, 1), dtype=torch.float64, device=rp.device)
    _check(lib().mgm_transpose(nrows, ncols, _p(rp), _p(ci), _p(v), _p(trp), _p(tci), _p(tv), _stream()))
    return trp, tci[:nnz], tv[:nnz]


def spgemm(nA, nB, ncolsB, a, b):
    arp, aci, av = a
    brp, bci, bv = b
    crp = torch.empty(nA + 1, dtype=torch.int32, device=arp.device)
    nnz = C.c_int64(0)
    L = lib()
    _check(L.mgm_spgemm(nA, nB, ncolsB, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv), _p(crp), None, None,
                        C.byref(nnz), _stream()))
    cci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=arp.device)
    cv = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=arp.device)
    _check(L.mgm_spgemm(nA, nB, ncolsB, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv), _p(crp), _p(cci), _p(cv),
                        C.byref(nnz), _stream()))
    return crp, cci[: nnz.value], cv[: nnz.value]


def rcm(rp, ci):
    N = rp.numel() - 1
    perm = torch.empty(N, dtype=torch.int32, device=rp.device)
    _check(lib().mgm_rcm(N, _p(rp), _p(ci), _p(perm), _stream()))
    return perm


def color(rp, ci, seed):
    N = rp.numel() - 1
    col = torch.empty(N, dtype=torch.int32, device=rp.device)
    nc = C.c_int32(0)
    _check(lib().mgm_color(N, _p(rp), _p(ci), seed, _p(col), C.byref(nc), _stream()))
    return col, nc.value


class Hierarchy:
    """MGM hierarchy (Alg. 2) owned by the library; V-cycle (Alg. 3) and FGMRES solve on it."""

    def __init__(self, xyz, rp, ci, v, n_min, m=3, nu1=1, nu2=1, precision="f32", seed=0, persistent_sweeps=5,
                 constraint=False, smoother="mc", cycle="V", transfer_bf16=False):
        """persistent_sweeps: how the multicolour sweeps are launched (mgm_params; default 5, staged
        per-colour launches; 0 one plain launch per colour; 4 autotuned per level).
        constraint=True: surface Poisson (L = D) with the mean-zero constraint of Sec. 4.4.
        smoother: "mc" multicolour Gauss-Seidel or "lex" lexicographic Gauss-Seidel (the paper's).
        cycle: "V" (Alg. 3), "W" or "F" (Sec. 4.5).
        transfer_bf16: the FP32 cycle reads its interpolation/restriction weights stored as BF16."""
        if smoother not in ("mc", "lex"):
            raise ValueError("smoother must be 'mc' or 'lex'")
        if cycle not in ("V", "W", "F"):
            raise ValueError("cycle must be 'V', 'W' or 'F'")
        xyz = _dev(xyz, torch.float64, "xyz"); rp = _dev(rp, torch.int32, "rowptr")
        ci = _dev(ci, torch.int32, "col"); v = _dev(v, torch.float64, "val")
        self.N = xyz.shape[0]
        self.device = xyz.device
        self.constraint = bool(constraint)
        prm = Params(n_min, m, nu1, nu2, MGM_F32 if precision == "f32" else MGM_F64, seed, int(persistent_sweeps),
                     int(constraint), 1 if smoother == "lex" else 0, {"V": 0, "W": 1, "F": 2}[cycle],
                     int(bool(transfer_bf16)))
        h = C.c_void_p()
        self._h = None
        _check(lib().mgm_setup(_p(xyz), self.N, _p(rp), _p(ci), _p(v), C.byref(prm), C.byref(h), _stream()))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().mgm_destroy(self._h)
            self._h = None

    def stats(self):
        s = HierStats()
        _check(lib().mgm_hierarchy_stats_get(self._h, C.byref(s)))
        p = s.p
        return {"p": p, "n": list(s.n[:p]), "nnz": list(s.nnz[:p]), "ncolors": list(s.ncolors[:p]),
                "device_bytes": s.device_bytes, "precision": "f32" if s.precision == MGM_F32 else "f64"}

    def level(self, j):
        st = self.stats()
        n, nnz = st["n"][j], st["nnz"][j]
        dev = self.device
        out = {"perm": torch.empty(n, dtype=torch.int32, device=dev),
               "xyz": torch.empty((n, 3), dtype=torch.float64, device=dev),
               "rp": torch.empty(n + 1, dtype=torch.int32, device=dev),
               "ci": torch.empty(nnz, dtype=torch.int32, device=dev),
               "v": torch.empty(nnz, dtype=torch.float64, device=dev)}
        keep = torch.empty(n, dtype=torch.int32, device=dev) if j >= 1 else None
        args = [None] * 6
        if j + 1 < st["p"]:
            pn = C.c_int64(0)
            _check(lib().mgm_hierarchy_pnnz(self._h, j, C.byref(pn)))
            out["prp"] = torch.empty(n + 1, dtype=torch.int32, device=dev)
            out["pci"] = torch.empty(pn.value, dtype=torch.int32, device=dev)
            out["pv"] = torch.empty(pn.value, dtype=torch.float64, device=dev)
            out["colour"] = torch.empty(n, dtype=torch.int32, device=dev)
            args = [out["prp"], out["pci"], out["pv"], out["colour"]]
        else:
            args = [None, None, None, None]
        _check(lib().mgm_hierarchy_level(self._h, j, _p(out["perm"]), _p(keep), _p(out["xyz"]), _p(out["rp"]),
                                         _p(out["ci"]), _p(out["v"]), *[_p(a) for a in args], _stream()))
        if keep is not None:
            out["keep"] = keep
        return out

    def profile(self, reps=20):
        """Device time and algorithmic bytes of one V-cycle, one finest-level sweep and one outer
        FP64 operator product (CUDA events; overwrites the hierarchy's work vectors)."""
        pi = ProfileInfo()
        _check(lib().mgm_profile(self._h, reps, C.byref(pi), _stream()))
        return {k: getattr(pi, k) for k, _ in ProfileInfo._fields_}

    def vcycle_floor(self, chain_us, gbs):
        """Lower bound (ms) of one V-cycle for colour-by-launch schedules (mgm_vcycle_floor):
        {"floor_ms", "bytes_ms", "chain_ms"}."""
        f, b, c = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
        _check(lib().mgm_vcycle_floor(self._h, chain_us, gbs, C.byref(f), C.byref(b), C.byref(c)))
        return {"floor_ms": f.value, "bytes_ms": b.value, "chain_ms": c.value}

    def sweep_config(self, level):
        """Sweep schedule of a level: {"kind": "launch"|"stream", "blocks", "lanes", "stages", "ms"}."""
        c = SweepConfig()
        _check(lib().mgm_sweep_config_get(self._h, level, C.byref(c)))
        return {"kind": _SCHEDULES[c.kind], "blocks": c.blocks, "lanes": c.lanes, "stages": c.stages, "ms": c.ms}

    def set_sweep_config(self, level, kind="stream", blocks=0, lanes=2, stages=2):
        """kind: "launch" (a kernel per colour), "stream" (one cooperative launch a sweep, progress
        counters), "resident" (one block holding the level's vector) or "colour" (a kernel per colour,
        each block's slice staged in shared memory before the programmatic-launch wait)."""
        c = SweepConfig(_SCHEDULES.index(kind), blocks, lanes, stages, 0.0)
        _check(lib().mgm_sweep_config_set(self._h, level, C.byref(c), _stream()))

    def profile_level(self, level, reps=10):
        """Device time (ms) of a level's smoothing work in one V-cycle under its current schedule."""
        ms = C.c_float(0.0)
        _check(lib().mgm_profile_level(self._h, level, reps, C.byref(ms), _stream()))
        return ms.value

    def tail_info(self):
        """(top level, cluster CTAs) of the cluster-resident coarse tail of the FP32 cycle; top 0: none."""
        t, c = C.c_int(0), C.c_int(0)
        _check(lib().mgm_tail_info(self._h, C.byref(t), C.byref(c)))
        return t.value, c.value

    def level_smoothing_bytes(self, level):
        """Algorithmic bytes of a level's smoothing work in one V-cycle (what profile_level times)."""
        b = C.c_int64(0)
        _check(lib().mgm_level_smoothing_bytes(self._h, level, C.byref(b)))
        return b.value

    def autotune(self, reps=5, use_cache=True):
        """Per-level choice of sweep schedule by timed trials (mgm_autotune); returns the choices."""
        _check(lib().mgm_autotune(self._h, reps, int(use_cache), _stream()))
        return [self.sweep_config(j) for j in range(self.stats()["p"] - 1)]

    def vcycle(self, r):
        if r.dtype not in (torch.float32, torch.float64):
            raise TypeError("r must be float32 or float64")
        r = _dev(r, r.dtype, "r")
        z = torch.empty_like(r)
        _check(lib().mgm_vcycle(self._h, _p(r), _p(z), MGM_F64 if r.dtype == torch.float64 else MGM_F32, _stream()))
        return z

    def solve(self, f, u0=None, krylov="fgmres", restart=50, maxit=200, tol=1e-10, raise_on_nonconv=False):
        f = _dev(f, torch.float64, "f")
        u = torch.zeros_like(f) if u0 is None else _dev(u0, torch.float64, "u0").clone()
        sp = SolveParams(_KRYLOV[krylov], restart, maxit, tol)
        hist = (C.c_double * (maxit + 2))()
        info = SolveInfo(0, 0.0, hist, maxit + 2, 0.0, 0.0)
        st = lib().mgm_solve(self._h, _p(f), _p(u), C.byref(sp), C.byref(info), _stream())
        if st != 0 and (st != 3 or raise_on_nonconv):
            _check(st)
        return u, {"iters": info.iters, "rel_res": info.rel_res, "solve_ms": info.solve_ms, "converged": st == 0,
                   "history": [hist[i] for i in range(info.iters + 1)], "multiplier": info.multiplier}


    def eigs(self, nev=16, block=8, steps=3, max_cycles=20, tol=1e-8, solve_tol=1e-10, restart=50, maxit=200,
             seed=0, vectors=True):
        """Eigenpairs of L of smallest magnitude by shift-invert (Sec. 6.1; see mgm_eigs). Returns
        (eigenvalues as complex numpy array, eigenvectors N x nev device tensor or None, info)."""
        import numpy as np
        N = self.stats()["n"][0]
        sp = SolveParams(_KRYLOV["fgmres"], restart, maxit, solve_tol)
        lr = (C.c_double * nev)(); li = (C.c_double * nev)(); rs = (C.c_double * nev)()
        vec = torch.empty((nev, N), dtype=torch.float64, device=self.device) if vectors else None
        nconv = C.c_int(0); nsol = C.c_int(0)
        _check(lib().mgm_eigs(self._h, nev, block, steps, max_cycles, tol, C.byref(sp), seed, lr, li, rs,
                              _p(vec) if vectors else None, C.byref(nconv), C.byref(nsol), _stream()))
        lam = np.array(lr[:]) + 1j * np.array(li[:])
        return lam, (vec.T if vectors else None), {"resid": list(rs[:]), "nconv": nconv.value, "solves": nsol.value}

    # ---- learned correction after the V-cycle (an addition to the paper's method)
    def learned_attach(self, xyz, nrm, idx, w):
        """Attach level-0 stencils (device tensors in caller order: xyz, nrm N x 3 float64, idx
        N x n int32 centre first, w N x n float64 LBO weights)."""
        xyz = _dev(xyz, torch.float64, "xyz"); nrm = _dev(nrm, torch.float64, "nrm")
        idx = _dev(idx, torch.int32, "idx"); w = _dev(w, torch.float64, "w")
        self.ln = idx.shape[1]
        _check(lib().mgm_learned_attach(self._h, _p(xyz), _p(nrm), _p(idx), _p(w), self.ln, _stream()))

    def learned_features(self, r):
        r = _dev(r, torch.float64, "r")
        feat = torch.empty((self.N, 4 * self.ln), dtype=torch.float32, device=r.device)
        rho = torch.empty(self.N, dtype=torch.float32, device=r.device)
        _check(lib().mgm_learned_features(self._h, _p(r), _p(feat), _p(rho), _stream()))
        return feat, rho

    def learned_cycle_residual(self, r):
        """r - L M r with the plain V-cycle M (a training sample)."""
        r = _dev(r, torch.float64, "r")
        out = torch.empty_like(r)
        _check(lib().mgm_learned_cycle_residual(self._h, _p(r), _p(out), _stream()))
        return out

    def learned_loss(self, net, r, grad=False):
        r = _dev(r, torch.float64, "r")
        J = C.c_double(0.0)
        g = torch.empty(net.size, dtype=torch.float32, device=r.device) if grad else None
        _check(lib().mgm_learned_loss(self._h, net._h, _p(r), C.byref(J), _p(g), _stream()))
        return (J.value, g) if grad else J.value

    def learned_train_step(self, net, r, lr):
        r = _dev(r, torch.float64, "r")
        J = C.c_double(0.0)
        _check(lib().mgm_learned_train_step(self._h, net._h, _p(r), float(lr), C.byref(J), _stream()))
        return J.value

    def learned_enable(self, net):
        """Use net (its current weights, BF16) after each V-cycle; None switches it off."""
        _check(lib().mgm_learned_enable(self._h, net._h if net is not None else None, _stream()))

    def learned_correction(self, r):
        r = _dev(r, torch.float64, "r")
        d = torch.empty_like(r)
        _check(lib().mgm_learned_correction(self._h, _p(r), _p(d), _stream()))
        return d

    def learned_info(self):
        en = C.c_int(0); fb = C.c_int64(0)
        _check(lib().mgm_learned_info(self._h, C.byref(en), C.byref(fb)))
        return {"enabled": bool(en.value), "fallbacks": int(fb.value)}


class MLP:
    """The learned correction's network (4n -> 64 -> 64 -> 1, no biases), owned by the library:
    FP32 master weights and Adam state on the device."""

    def __init__(self, n, seed=0):
        self.n = n
        self.size = int(lib().mgm_mlp_size(n))
        if self.size < 0:
            raise ValueError("stencil size must be in [1, 48]")
        h = C.c_void_p()
        self._h = None
        _check(lib().mgm_mlp_create(n, seed, C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().mgm_mlp_destroy(self._h)
            self._h = None

    def get(self):
        """(W1 64 x 4n, W2 64 x 64, w3 64) as float32 numpy arrays."""
        import numpy as np
        w = np.empty(self.size, np.float32)
        _check(lib().mgm_mlp_get(self._h, w.ctypes.data))
        d = 4 * self.n
        return w[:64 * d].reshape(64, d).copy(), w[64 * d:64 * d + 4096].reshape(64, 64).copy(), w[64 * d + 4096:].copy()

    def set(self, W1, W2, w3):
        import numpy as np
        w = np.ascontiguousarray(np.concatenate([np.ravel(W1), np.ravel(W2), np.ravel(w3)]).astype(np.float32))
        if w.size != self.size:
            raise ValueError("weight shapes do not match the stencil size")
        _check(lib().mgm_mlp_set(self._h, w.ctypes.data))

    def forward(self, feat):
        feat = _dev(feat, torch.float32, "feat")
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(lib().mgm_mlp_forward(self._h, _p(feat), feat.shape[0], _p(out), _stream()))
        return out

    def vjp(self, feat, gout):
        feat = _dev(feat, torch.float32, "feat"); gout = _dev(gout, torch.float32, "gout")
        g = torch.empty(self.size, dtype=torch.float32, device=feat.device)
        _check(lib().mgm_mlp_vjp(self._h, _p(feat), _p(gout), feat.shape[0], _p(g), _stream()))
        d = 4 * self.n
        return g[:64 * d].reshape(64, d), g[64 * d:64 * d + 4096].reshape(64, 64), g[64 * d + 4096:]


def check_bounded_wait(nblocks=4, spin_limit=20000):
    """Run a device barrier that cannot complete; returns the status the library reports
    (MGM_ERR_TIMEOUT = 5 when the bounded wait gave up as designed)."""
    st = C.c_int(-1)
    _check(lib().mgm_check_bounded_wait(nblocks, spin_limit, C.byref(st), _stream()))
    return st.value


def kernel_launches():
    """Kernels launched by libmgm so far in this process."""
    return int(lib().mgm_kernel_launches())


def _multi_infos(nrhs, maxit):
    hists = [(C.c_double * (maxit + 2))() for _ in range(nrhs)]
    infos = (SolveInfo * nrhs)()
    for r in range(nrhs):
        infos[r] = SolveInfo(0, 0.0, hists[r], maxit + 2, 0.0, 0.0)
    return infos, hists


def _info_dicts(infos, hists, st, nrhs):
    return [{"iters": infos[r].iters, "rel_res": infos[r].rel_res, "solve_ms": infos[r].solve_ms,
             "converged": st == 0 or infos[r].rel_res <= 0.0,
             "history": [hists[r][i] for i in range(infos[r].iters + 1)]} for r in range(nrhs)]


def solve_multi(H, F, U0=None, krylov="fgmres", restart=50, maxit=200, tol=1e-10):
    """mgm_solve_multi: F is (nrhs, N) float64 CUDA (row r = right-hand side r); returns (U, infos)."""
    F = _dev(F, torch.float64, "F")
    nrhs = F.shape[0]
    U = torch.zeros_like(F) if U0 is None else _dev(U0, torch.float64, "U0").clone()
    sp = SolveParams(MGM_KRYLOV_FGMRES if krylov == "fgmres" else MGM_KRYLOV_NONE, restart, maxit, tol)
    infos, hists = _multi_infos(nrhs, maxit)
    st = lib().mgm_solve_multi(H._h, nrhs, _p(F), _p(U), C.byref(sp), infos, _stream())
    if st not in (0, 3):
        _check(st)
    out = _info_dicts(infos, hists, st, nrhs)
    for r in range(nrhs):
        out[r]["converged"] = infos[r].rel_res <= tol
    return U, out


def solve_batched(Hs, Fs, krylov="fgmres", restart=50, maxit=200, tol=1e-10):
    """mgm_solve_batched over problems q (hierarchy Hs[q], right-hand sides Fs[q] of shape (nrhs, N_q))."""
    nprob = len(Hs)
    nrhs = Fs[0].shape[0]
    Fs = [_dev(F, torch.float64, "F") for F in Fs]
    Us = [torch.zeros_like(F) for F in Fs]
    hp = (C.c_void_p * nprob)(*[H._h for H in Hs])
    fp = (C.c_void_p * nprob)(*[F.data_ptr() for F in Fs])
    up = (C.c_void_p * nprob)(*[U.data_ptr() for U in Us])
    sp = SolveParams(MGM_KRYLOV_FGMRES if krylov == "fgmres" else MGM_KRYLOV_NONE, restart, maxit, tol)
    infos, hists = _multi_infos(nprob * nrhs, maxit)
    status = (C.c_int * nprob)()
    st = lib().mgm_solve_batched(hp, nprob, fp, up, nrhs, C.byref(sp), infos, status, _stream())
    if st not in (0, 3):
        _check(st)
    out = _info_dicts(infos, hists, st, nprob * nrhs)
    for q in range(nprob * nrhs):
        out[q]["converged"] = infos[q].rel_res <= tol
        out[q]["status"] = STATUS.get(status[q // nrhs], status[q // nrhs])
    return Us, [out[q * nrhs:(q + 1) * nrhs] for q in range(nprob)]


def solve_points(xyz, nrm, f, n, method="rbf", k=1, ell=2, mu=1.0, alpha=4.0, n_min=250, m=3, precision="f32",
                 tol=1e-10, restart=50, maxit=200, seed=0):
    """The whole path from a point cloud to a solution: stencils (Sec. 2), hierarchy (Alg. 2),
    MGM-preconditioned FGMRES (Sec. 4.6). Inputs are CUDA tensors; returns (u, info, hierarchy)."""
    _, _, rp, ci, v = build_stencils(xyz, nrm, n, method, k, ell, mu, alpha, keep_weights=False)
    H = Hierarchy(xyz, rp, ci, v, n_min, m=m, precision=precision, seed=seed)
    u, info = H.solve(f, tol=tol, restart=restart, maxit=maxit)
    return u, info, H
