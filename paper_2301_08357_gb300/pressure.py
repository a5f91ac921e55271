"""Python binding of libpressure's C ABI (include/pressure.h).

Argument marshalling only: every function has the C function's name, converts
numpy arrays / torch tensors / ints to pointers, and calls the library.  Every
step of the computation runs in the CUDA library; there is no fallback.  If
libpressure.so is missing, importing this module raises.

Negative statuses raise PressureError, except the "soft" outcomes a caller is
expected to inspect (PS_ENOTCONV, PS_EBREAKDOWN, PS_PENDING), which are
returned together with the filled info struct.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpressure.so")

PS_OK, PS_PENDING = 0, 1
PS_EINVAL, PS_ENOMEM, PS_ENOTCONV, PS_EBREAKDOWN = -1, -2, -3, -4
PS_ETIMEOUT, PS_ECUDA, PS_ESTATE, PS_ENOTFOUND = -5, -6, -7, -8
PS_F32, PS_F64 = 1, 2
PS_MODE_FP64, PS_MODE_MIXED = 0, 1
PS_PRECOND_NONE, PS_PRECOND_JACOBI = 0, 1
PS_ENGINE_AUTO, PS_ENGINE_GRAPH, PS_ENGINE_PERSISTENT, PS_ENGINE_FUSED = 0, 1, 2, 3
PS_MASS_CONSISTENT, PS_MASS_LUMPED = 0, 1
SOFT = {PS_OK, PS_PENDING, PS_ENOTCONV, PS_EBREAKDOWN}


class PressureError(RuntimeError):
    def __init__(self, status, where):
        msg = "%s failed: %s (%d)" % (where, ps_status_str(status), status)
        try:
            detail = _lib.ps_last_error().decode()
            if detail:
                msg += ": " + detail
        except Exception:
            pass
        super().__init__(msg)
        self.status = status


class ps_mesh_opts(C.Structure):
    _fields_ = [("chunk_elems", C.c_int32), ("chunk_nodes_max", C.c_int32), ("pipeline", C.c_int32),
                ("update_blocks_per_sm", C.c_int32), ("operator_kernel", C.c_int32),
                ("operator_threads", C.c_int32), ("split_lead", C.c_int32), ("reserved", C.c_int32 * 1)]


class ps_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int64), ("mode", C.c_int32), ("precond", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("graph_iters", C.c_int32),
                ("engine", C.c_int32), ("grid_spin_limit", C.c_int32), ("batch_threads", C.c_int32),
                ("batch_order", C.c_int32), ("reserved", C.c_int32 * 2)]


class ps_projection_opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("dt", C.c_double), ("n_picard", C.c_int32),
                ("reserved", C.c_int32 * 7), ("solve", ps_solve_opts)]


class ps_solve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("converged", C.c_int32), ("iters_outer", C.c_int64),
                ("iters_inner", C.c_int64), ("rel_res", C.c_double), ("bnorm", C.c_double),
                ("n_free", C.c_int64), ("seconds", C.c_double), ("kernel_launches", C.c_int64),
                ("queue_seconds", C.c_double), ("reserved", C.c_double * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ps_mesh_stats(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_free", C.c_int64), ("dim", C.c_int32),
                ("n_chunks", C.c_int32), ("n_shared", C.c_int64), ("chunk_node_refs", C.c_int64),
                ("device_bytes", C.c_int64), ("max_chunk_elems", C.c_int32), ("max_chunk_nodes", C.c_int32),
                ("solve_bytes", C.c_int64), ("operator_kernel", C.c_int64), ("reserved", C.c_int64 * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ps_server_opts(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("epoch_iters", C.c_int32), ("hbm_budget_bytes", C.c_size_t),
                ("opts", ps_solve_opts), ("single_nodes", C.c_int32), ("reserved", C.c_int32 * 7)]


class ps_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("in_flight", C.c_int64), ("queued", C.c_int64), ("epochs", C.c_int64),
                ("peak_in_flight", C.c_int64), ("bytes_in_use", C.c_int64), ("busy_seconds", C.c_double),
                ("single_solves", C.c_int64), ("reserved", C.c_int64 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ps_eos_opts(C.Structure):
    _fields_ = [("eos_a", C.c_double), ("eos_b", C.c_double), ("dt", C.c_double), ("n_picard", C.c_int32),
                ("max_newton", C.c_int32), ("newton_tol", C.c_double), ("reserved", C.c_double * 4),
                ("solve", ps_solve_opts)]


_vp, _i64, _i32, _dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)

# name -> (restype, argtypes); mirrors include/pressure.h plus the debug hooks.
SIGNATURES = {
    "ps_version": (C.c_char_p, []),
    "ps_status_str": (C.c_char_p, [C.c_int]),
    "ps_last_error": (C.c_char_p, []),
    "ps_ctx_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_size_t]),
    "ps_ctx_destroy": (None, [_vp]),
    "ps_ctx_bytes_in_use": (_i64, [_vp]),
    "ps_mesh_upload": (C.c_int, [_vp, C.c_int, _i64, _vp, _i64, _vp, _vp, C.POINTER(ps_mesh_opts),
                                 C.POINTER(_vp)]),
    "ps_mesh_upload_periodic": (C.c_int, [_vp, C.c_int, _i64, _vp, _i64, _vp, _vp, _vp, C.POINTER(ps_mesh_opts),
                                 C.POINTER(_vp)]),
    "ps_mesh_free": (None, [_vp]),
    "ps_mesh_get_stats": (C.c_int, [_vp, C.POINTER(ps_mesh_stats)]),
    "ps_coeff_set": (C.c_int, [_vp, _vp, _vp, C.c_double]),
    "ps_coeff_set_beta": (C.c_int, [_vp, _vp]),
    "ps_pressure_apply": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ps_pressure_apply_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ps_pressure_solve": (C.c_int, [_vp, _vp, _vp, C.POINTER(ps_solve_opts), C.POINTER(ps_solve_info), _vp]),
    "ps_projection_opts_default": (None, [C.POINTER(ps_projection_opts)]),
    "ps_projection_step": (C.c_int, [_vp, C.POINTER(ps_projection_opts), _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp, C.POINTER(ps_solve_info), _vp]),
    "ps_mesh_set_mass": (C.c_int, [_vp, C.c_int]),
    "ps_eos_opts_default": (None, [C.POINTER(ps_eos_opts)]),
    "ps_projection_step_eos": (C.c_int, [_vp, C.POINTER(ps_eos_opts), _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                         _vp, _vp, _vp, C.POINTER(ps_solve_info), _vp]),
    "ps_solve_opts_default": (None, [C.POINTER(ps_solve_opts)]),
    "ps_batch_solve": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp),
                                 C.POINTER(ps_solve_opts), C.POINTER(ps_solve_info), _vp]),
    "ps_server_create": (C.c_int, [_vp, C.POINTER(ps_server_opts), C.POINTER(_vp)]),
    "ps_server_destroy": (None, [_vp]),
    "ps_server_add_case": (C.c_int, [_vp, _vp, _vp, C.POINTER(_i32)]),
    "ps_solve_submit": (C.c_int, [_vp, _i32, _vp, _vp, C.POINTER(_i64)]),
    "ps_solve_poll": (C.c_int, [_vp, _i64, C.POINTER(ps_solve_info), _vp]),
    "ps_solve_wait": (C.c_int, [_vp, _i64, C.c_double, C.POINTER(ps_solve_info), _vp]),
    "ps_server_release": (C.c_int, [_vp, _i64]),
    "ps_server_get_stats": (C.c_int, [_vp, C.POINTER(ps_server_stats)]),
    "ps_profile_kernel": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.POINTER(C.c_double)]),
    "ps_mesh_get_jacobi": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "ps_debug_cg_apply": (C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_double), _vp]),
    "ps_debug_prepare": (C.c_int, [C.c_int, _i64, _vp, _i64, _vp, _vp, _vp, C.POINTER(ps_mesh_opts),
                                   C.POINTER(ps_mesh_stats)]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpressure.so is not built (run __graft_entry__.build() or "
                          "python -m paper_2301_08357_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


# ---------------------------------------------------------------- marshalling
def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_vp)


def _dev(t):
    """Device pointer of a torch tensor (or an int address)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("device tensor must be contiguous")
        return _vp(t.data_ptr())
    return _vp(int(t))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return _vp(s.cuda_stream)
    return _vp(int(s))


def _check(status, where):
    if status not in SOFT:
        raise PressureError(status, where)
    return status


# ---------------------------------------------------------------- API (same names as C)
def ps_version():
    return _lib.ps_version().decode()


def ps_status_str(status):
    return _lib.ps_status_str(int(status)).decode()


def ps_ctx_create(device=0, hbm_budget_bytes=0):
    h = _vp()
    _check(_lib.ps_ctx_create(C.byref(h), int(device), int(hbm_budget_bytes)), "ps_ctx_create")
    return h


def ps_ctx_destroy(ctx):
    _lib.ps_ctx_destroy(ctx)


def ps_ctx_bytes_in_use(ctx):
    return int(_lib.ps_ctx_bytes_in_use(ctx))


def ps_mesh_upload(ctx, dim, coords, conn, dirichlet=None, chunk_elems=0, chunk_nodes_max=0, pipeline=0,
                   update_blocks_per_sm=0, periodic=None, operator_kernel=0, operator_threads=0, split_lead=0):
    """periodic: optional [n_nodes] master map (ps_mesh_upload_periodic)."""
    coords, pc = _host(coords, np.float64)
    conn, pe = _host(conn, np.int32)
    n = coords.shape[0]
    pd = None
    if dirichlet is not None:
        dirichlet, pd = _host(dirichlet, np.uint8)
    o = ps_mesh_opts(chunk_elems, chunk_nodes_max, pipeline, update_blocks_per_sm, operator_kernel,
                     operator_threads, split_lead)
    h = _vp()
    if periodic is None:
        _check(_lib.ps_mesh_upload(ctx, int(dim), n, pc, conn.shape[0], pe, pd, C.byref(o), C.byref(h)),
               "ps_mesh_upload")
    else:
        periodic, pp = _host(periodic, np.int32)
        _check(_lib.ps_mesh_upload_periodic(ctx, int(dim), n, pc, conn.shape[0], pe, pd, pp, C.byref(o),
                                            C.byref(h)), "ps_mesh_upload_periodic")
    return h


def ps_mesh_free(mesh):
    _lib.ps_mesh_free(mesh)


def ps_mesh_get_stats(mesh):
    s = ps_mesh_stats()
    _check(_lib.ps_mesh_get_stats(mesh, C.byref(s)), "ps_mesh_get_stats")
    return s


def ps_coeff_set(mesh, alpha, beta, dt2):
    alpha, pa = _host(alpha, np.float64)
    beta, pb = _host(beta, np.float64)
    return _check(_lib.ps_coeff_set(mesh, pa, pb, float(dt2)), "ps_coeff_set")


def ps_coeff_set_beta(mesh, beta):
    beta, pb = _host(beta, np.float64)
    return _check(_lib.ps_coeff_set_beta(mesh, pb), "ps_coeff_set_beta")


def ps_pressure_apply(mesh, x_dev, y_dev, precision, stream=None):
    return _check(_lib.ps_pressure_apply(mesh, _dev(x_dev), _dev(y_dev), int(precision), _stream(stream)),
                  "ps_pressure_apply")


def ps_pressure_apply_noalloc(mesh, x_dev, y_dev, precision, stream=None):
    """Apply without any device allocation (scratch in a fixed 16 MiB device array)."""
    return _check(_lib.ps_pressure_apply_noalloc(mesh, _dev(x_dev), _dev(y_dev), int(precision), _stream(stream)),
                  "ps_pressure_apply_noalloc")


def ps_solve_opts_default():
    o = ps_solve_opts()
    _lib.ps_solve_opts_default(C.byref(o))
    return o


def make_opts(**kw):
    o = ps_solve_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ps_pressure_solve(mesh, b_dev, x_dev, opts=None, stream=None):
    """Returns (status, info)."""
    info = ps_solve_info()
    o = C.byref(opts) if opts is not None else None
    st = _lib.ps_pressure_solve(mesh, _dev(b_dev), _dev(x_dev), o, C.byref(info), _stream(stream))
    return _check(st, "ps_pressure_solve"), info


def ps_projection_opts_default():
    o = ps_projection_opts()
    _lib.ps_projection_opts_default(C.byref(o))
    return o


def ps_projection_step(mesh, rho, wu, we, pn, dp, p_out, wu_out, h_out, rhok_out, gamma=1.4, dt=None,
                       n_picard=2, solve_opts=None, stream=None):
    """One time step's projection stage (device arrays, caller's numbering /
    element order; dp is the first guess in and dP out).  Returns (status, info)."""
    o = ps_projection_opts_default()
    o.gamma = float(gamma)
    o.dt = float(dt) if dt is not None else 0.0
    o.n_picard = int(n_picard)
    if solve_opts is not None:
        o.solve = solve_opts
    info = ps_solve_info()
    st = _lib.ps_projection_step(mesh, C.byref(o), _dev(rho), _dev(wu), _dev(we), _dev(pn), _dev(dp), _dev(p_out),
                                 _dev(wu_out), _dev(h_out), _dev(rhok_out), C.byref(info), _stream(stream))
    return _check(st, "ps_projection_step"), info


def ps_mesh_set_mass(mesh, mass):
    """PS_MASS_CONSISTENT or PS_MASS_LUMPED (vertex-quadrature mass)."""
    return _check(_lib.ps_mesh_set_mass(mesh, int(mass)), "ps_mesh_set_mass")


def ps_eos_opts_default():
    o = ps_eos_opts()
    _lib.ps_eos_opts_default(C.byref(o))
    return o


def ps_projection_step_eos(mesh, rho, wu, we, pn, dp, p_out, wu_out, h_out, rhok_out, eos_a=2.5, eos_b=0.0,
                           dt=None, n_picard=2, max_newton=8, newton_tol=1e-8, solve_opts=None, stream=None):
    """Projection stage with rho e = eos_a P + eos_b P^2 / rho, lumped mass and
    Newton's method per Picard iteration.  Returns (status, info, res) with
    res[k, j] = ||F|| / ||c|| at Newton check j of Picard iteration k (-1:
    no check)."""
    o = ps_eos_opts_default()
    o.eos_a, o.eos_b = float(eos_a), float(eos_b)
    o.dt = float(dt) if dt is not None else 0.0
    o.n_picard, o.max_newton, o.newton_tol = int(n_picard), int(max_newton), float(newton_tol)
    if solve_opts is not None:
        o.solve = solve_opts
    res = np.full((max(int(n_picard), 1), max(int(max_newton), 0) + 1), -1.0)
    info = ps_solve_info()
    st = _lib.ps_projection_step_eos(mesh, C.byref(o), _dev(rho), _dev(wu), _dev(we), _dev(pn), _dev(dp),
                                     _dev(p_out), _dev(wu_out), _dev(h_out), _dev(rhok_out),
                                     res.ctypes.data_as(_vp), C.byref(info), _stream(stream))
    return _check(st, "ps_projection_step_eos"), info, res


def ps_batch_solve(meshes, b_devs, x_devs, opts=None, stream=None):
    """Returns (status, [info ...])."""
    n = len(meshes)
    M = (_vp * n)(*meshes)
    B = (_vp * n)(*[_dev(b).value for b in b_devs])
    X = (_vp * n)(*[_dev(x).value for x in x_devs])
    infos = (ps_solve_info * n)()
    o = C.byref(opts) if opts is not None else None
    st = _lib.ps_batch_solve(M, n, B, X, o, infos, _stream(stream))
    return _check(st, "ps_batch_solve"), list(infos)


def ps_server_create(ctx, max_slots=0, epoch_iters=0, hbm_budget_bytes=0, opts=None, single_nodes=0):
    so = ps_server_opts()
    so.max_slots, so.epoch_iters, so.hbm_budget_bytes = max_slots, epoch_iters, hbm_budget_bytes
    so.single_nodes = single_nodes
    so.opts = opts if opts is not None else ps_solve_opts_default()
    h = _vp()
    _check(_lib.ps_server_create(ctx, C.byref(so), C.byref(h)), "ps_server_create")
    return h


def ps_server_destroy(srv):
    _lib.ps_server_destroy(srv)


def ps_server_add_case(srv, mesh, x0=None):
    px = None
    if x0 is not None:
        x0, px = _host(x0, np.float64)
    cid = _i32()
    _check(_lib.ps_server_add_case(srv, mesh, px, C.byref(cid)), "ps_server_add_case")
    return int(cid.value)


def ps_solve_submit(srv, case_id, b, beta=None):
    b, pb = _host(b, np.float64)
    pbeta = None
    if beta is not None:
        beta, pbeta = _host(beta, np.float64)
    t = _i64()
    _check(_lib.ps_solve_submit(srv, int(case_id), pb, pbeta, C.byref(t)), "ps_solve_submit")
    return int(t.value)


def ps_solve_poll(srv, ticket, x_out=None):
    """Returns (status, info); x_out (host float64 array) is filled when done."""
    info = ps_solve_info()
    px = None
    if x_out is not None:
        assert x_out.dtype == np.float64 and x_out.flags.c_contiguous
        px = x_out.ctypes.data_as(_vp)
    st = _lib.ps_solve_poll(srv, int(ticket), C.byref(info), px)
    return _check(st, "ps_solve_poll"), info


def ps_solve_wait(srv, ticket, timeout_s=600.0, x_out=None):
    info = ps_solve_info()
    px = None
    if x_out is not None:
        assert x_out.dtype == np.float64 and x_out.flags.c_contiguous
        px = x_out.ctypes.data_as(_vp)
    st = _lib.ps_solve_wait(srv, int(ticket), float(timeout_s), C.byref(info), px)
    return _check(st, "ps_solve_wait"), info


def ps_server_release(srv, ticket):
    return _check(_lib.ps_server_release(srv, int(ticket)), "ps_server_release")


def ps_server_get_stats(srv):
    s = ps_server_stats()
    _check(_lib.ps_server_get_stats(srv, C.byref(s)), "ps_server_get_stats")
    return s


PS_KERNEL_CG_F32, PS_KERNEL_UPDATE_F32, PS_KERNEL_APPLY_F32, PS_KERNEL_RESID_F64, PS_KERNEL_CG_F64 = 0, 1, 2, 3, 4
PS_KERNEL_CG1_F32 = 5
PS_KERNEL_HALO_F32 = 6


def ps_profile_kernel(mesh, which, reps=20, stream=None):
    """Average device ms per launch of one internal kernel (CUDA events on `stream`)."""
    ms = C.c_double()
    _check(_lib.ps_profile_kernel(mesh, int(which), int(reps), _stream(stream), C.byref(ms)), "ps_profile_kernel")
    return float(ms.value)


def ps_mesh_get_jacobi(mesh, precision=PS_F64, stream=None):
    """The Jacobi preconditioner's inverse diagonal, caller numbering (host
    NumPy array, float64 or float32)."""
    n = ps_mesh_get_stats(mesh).n_nodes
    out = np.empty(n, dtype=np.float64 if precision == PS_F64 else np.float32)
    _check(_lib.ps_mesh_get_jacobi(mesh, int(precision), out.ctypes.data_as(C.c_void_p), _stream(stream)),
           "ps_mesh_get_jacobi")
    return out


def ps_debug_cg_apply(mesh, x_dev, y_dev, stream=None):
    """One pass of the FP32 CG operator kernel with direction x: fills y = A x
    (device float tensors) and returns x^T A x as the kernel accumulates it."""
    pap = C.c_double()
    _check(_lib.ps_debug_cg_apply(mesh, _dev(x_dev), _dev(y_dev), C.byref(pap), _stream(stream)),
           "ps_debug_cg_apply")
    return float(pap.value)


def ps_debug_prepare(dim, coords, conn, dirichlet=None, chunk_elems=0, chunk_nodes_max=0, periodic=None,
                     split_lead=0):
    """Host-only: run the mesh preprocessing and its invariant checks."""
    coords, pc = _host(coords, np.float64)
    conn, pe = _host(conn, np.int32)
    pd = None
    if dirichlet is not None:
        dirichlet, pd = _host(dirichlet, np.uint8)
    pp = None
    if periodic is not None:
        periodic, pp = _host(periodic, np.int32)
    o = ps_mesh_opts(chunk_elems, chunk_nodes_max)
    o.split_lead = split_lead
    s = ps_mesh_stats()
    _check(_lib.ps_debug_prepare(int(dim), coords.shape[0], pc, conn.shape[0], pe, pd, pp, C.byref(o),
                                 C.byref(s)), "ps_debug_prepare")
    return s
