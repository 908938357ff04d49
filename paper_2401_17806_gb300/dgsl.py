"""ctypes binding of the dgsl C-ABI (``include/dgsl.h``).

Argument marshalling only: every computation runs in ``libdgsl.so``.
Device vectors are passed as PyTorch CUDA tensors (their ``data_ptr()``),
streams as ``torch.cuda.Stream`` (their ``cuda_stream`` handle) or None for
the current stream.  If the library has not been built this module raises on
first use; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- constants
OK, EINVAL, EMESH, ENOMEM, EBUDGET, ENOTCONV, ETIMEOUT, EPENDING, ECUDA, ENODEVICE = range(10)
STORE_F64, STORE_F32, STORE_BF16 = 1, 2, 4
MAIN, DUAL = 0, 1
FORM_ASSEMBLED, FORM_FACTORED = 0, 1
SCHUR, HELMHOLTZ = 0, 1
PREC_F64, PREC_F32_IR, PREC_BF16_IR = 0, 1, 2
PRECOND_NONE, PRECOND_BLOCK_JACOBI, PRECOND_MULTIGRID = 0, 1, 2


class DgslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dgsl error {code}: {msg}")
        self.code = code


class dgsl_mesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("xy", C.POINTER(C.c_double)),
                ("n_triangles", C.c_int32), ("tri", C.POINTER(C.c_int32)),
                ("period", C.c_double * 2)]


class dgsl_build_opts(C.Structure):
    _fields_ = [("host_only", C.c_int32), ("device", C.c_int32), ("store", C.c_int32),
                ("factored", C.c_int32), ("stream", C.c_void_p)]


class dgsl_info(C.Structure):
    _fields_ = [("p", C.c_int32), ("n_phi", C.c_int32), ("n_psi", C.c_int32),
                ("n_tri", C.c_int32), ("n_edge", C.c_int32), ("n_colours", C.c_int32),
                ("n_dof", C.c_int64), ("n_dual", C.c_int64), ("device_bytes", C.c_int64),
                ("host_only", C.c_int32), ("device", C.c_int32)]


class dgsl_maps(C.Structure):
    _fields_ = [("edge_vtx", C.c_void_p), ("lr", C.c_void_p), ("loc", C.c_void_p),
                ("shift", C.c_void_p), ("tri_edge", C.c_void_p), ("perm", C.c_void_p),
                ("edge_perm", C.c_void_p), ("colour", C.c_void_p),
                ("colour_offsets", C.c_void_p)]


class dgsl_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int32), ("precision", C.c_int32),
                ("use_x0", C.c_int32), ("inner_tol", C.c_double), ("max_refine", C.c_int32),
                ("form", C.c_int32), ("precond", C.c_int32), ("pad", C.c_int32)]


class dgsl_solve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("refinements", C.c_int32),
                ("cg_launches", C.c_int32), ("relres", C.c_double), ("cg_kernel_ms", C.c_double),
                ("grid", C.c_int32), ("pad", C.c_int32), ("relres_floor", C.c_double)]


MAX_RHS = 8  # right-hand sides per engine request


class dgsl_mg_info(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_vertices", C.c_int32), ("sizes", C.c_int32 * 16)]


class dgsl_request(C.Structure):
    _fields_ = [("op", C.c_void_p), ("kind", C.c_int32), ("n_rhs", C.c_int32), ("coef", C.c_double),
                ("b", C.c_void_p), ("x", C.c_void_p), ("tol", C.c_double)]


class dgsl_engine_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iters", C.c_int32), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("device", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("idle_us", C.c_int64), ("precond", C.c_int32), ("pad", C.c_int32)]


class dgsl_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64),
                ("in_flight", C.c_int64), ("engine_launches", C.c_int64), ("bytes_in_use", C.c_int64),
                ("admitted_running", C.c_int64)]


_LIB = None

_SIGS = {
    "dgsl_last_error": (C.c_char_p, []),
    "dgsl_version": (C.c_char_p, []),
    "dgsl_launch_count": (C.c_uint64, []),
    "dgsl_build_operators": (C.c_int, [C.POINTER(dgsl_mesh), C.c_int, C.POINTER(dgsl_build_opts),
                                       C.POINTER(C.c_void_p)]),
    "dgsl_destroy_operator": (None, [C.c_void_p]),
    "dgsl_operator_info": (C.c_int, [C.c_void_p, C.POINTER(dgsl_info)]),
    "dgsl_query_maps": (C.c_int, [C.c_void_p, C.POINTER(dgsl_maps)]),
    "dgsl_node_coords": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dgsl_query_blocks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgsl_apply_schur": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                   C.c_int, C.c_void_p]),
    "dgsl_apply_schur_f32": (C.c_int, [C.c_void_p, C.c_float, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_void_p]),
    "dgsl_apply_helmholtz": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_void_p]),
    "dgsl_project_d2m_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dgsl_project_m2d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dgsl_apply_div": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dgsl_velocity_update": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_void_p]),
    "dgsl_sl_quadrature": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "dgsl_ns_step": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(dgsl_solve_opts), C.POINTER(dgsl_solve_info), C.c_void_p]),
    "dgsl_query_sl_tables": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgsl_sl_transport": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgsl_sl_transport_imex": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgsl_ns_imex_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(dgsl_solve_opts), C.POINTER(dgsl_solve_info),
                                    C.c_void_p]),
    "dgsl_advdiff_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(dgsl_solve_opts), C.POINTER(dgsl_solve_info),
                                    C.c_void_p]),
    "dgsl_cg_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_int,
                                C.POINTER(dgsl_solve_opts), C.POINTER(dgsl_solve_info), C.c_void_p]),
    "dgsl_default_solve_opts": (None, [C.POINTER(dgsl_solve_opts)]),
    "dgsl_default_engine_opts": (None, [C.POINTER(dgsl_engine_opts)]),
    "dgsl_selftest_wait_timeout": (C.c_int, [C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)]),
    "dgsl_measure_fma_rate": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "dgsl_query_couplings": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dgsl_cg_solve_batch": (C.c_int, [C.POINTER(dgsl_request), C.c_int, C.POINTER(dgsl_engine_opts),
                                      C.POINTER(dgsl_solve_info), C.c_void_p]),
    "dgsl_server_create": (C.c_int, [C.POINTER(dgsl_engine_opts), C.POINTER(C.c_void_p)]),
    "dgsl_submit": (C.c_int, [C.c_void_p, C.POINTER(dgsl_request), C.POINTER(C.c_uint64)]),
    "dgsl_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(dgsl_solve_info)]),
    "dgsl_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "dgsl_poll_many": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dgsl_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(dgsl_server_stats)]),
    "dgsl_server_destroy": (None, [C.c_void_p]),
    "dgsl_apply_multigrid": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "dgsl_query_multigrid": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(dgsl_mg_info), C.c_void_p,
                                       C.c_void_p]),
    "dgsl_cg_solve_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                        C.c_int, C.POINTER(dgsl_solve_opts),
                                        C.POINTER(dgsl_solve_info), C.c_void_p]),
}


def library_path():
    return _build.LIB


def load():
    """Load libdgsl.so (built in-tree by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(code):
    if code != OK:
        raise DgslError(code, load().dgsl_last_error().decode())
    return code


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dptr(t, dtype_name, numel):
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    if str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"{dtype_name} tensor expected, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"tensor has {t.numel()} elements, expected {numel}")
    return C.c_void_p(t.data_ptr())


def dgsl_version():
    return load().dgsl_version().decode()


def dgsl_launch_count():
    return int(load().dgsl_launch_count())


def dgsl_default_solve_opts():
    o = dgsl_solve_opts()
    load().dgsl_default_solve_opts(C.byref(o))
    return o


class Operator:
    """Owning handle of one built operator (``dgsl_build_operators``)."""

    def __init__(self, xy, tri, period, p, host_only=False, device=0, store=0, factored=False, stream=None):
        lib = load()
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32)
        m = dgsl_mesh(self._xy.shape[0], self._xy.ctypes.data_as(C.POINTER(C.c_double)),
                      self._tri.shape[0], self._tri.ctypes.data_as(C.POINTER(C.c_int32)),
                      (C.c_double * 2)(float(period[0]), float(period[1])))
        o = dgsl_build_opts(int(host_only), int(device), int(store), int(factored),
                            _stream(stream).value if stream is not None else None)
        h = C.c_void_p()
        _check(lib.dgsl_build_operators(C.byref(m), int(p), C.byref(o), C.byref(h)))
        self.h = h
        inf = dgsl_info()
        _check(lib.dgsl_operator_info(self.h, C.byref(inf)))
        self.p = inf.p
        self.n_phi, self.n_psi = inf.n_phi, inf.n_psi
        self.n_tri, self.n_edge, self.n_colours = inf.n_tri, inf.n_edge, inf.n_colours
        self.n_dof, self.n_dual = inf.n_dof, inf.n_dual
        self.device_bytes = inf.device_bytes
        self.device = inf.device

    def close(self):
        if getattr(self, "h", None):
            load().dgsl_destroy_operator(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host queries
    def maps(self):
        ne, nd = self.n_tri, self.n_edge
        out = dict(edge_vtx=np.zeros((nd, 2), np.int32), lr=np.zeros((nd, 2), np.int32),
                   loc=np.zeros((nd, 2), np.uint8), shift=np.zeros((nd, 2), np.int8),
                   tri_edge=np.zeros((ne, 3), np.int32), perm=np.zeros(ne, np.int32),
                   edge_perm=np.zeros(nd, np.int32), colour=np.zeros(nd, np.uint8),
                   colour_offsets=np.zeros(self.n_colours + 1, np.int32))
        m = dgsl_maps(*[C.c_void_p(out[f].ctypes.data) for f, _ in dgsl_maps._fields_])
        _check(load().dgsl_query_maps(self.h, C.byref(m)))
        return out

    def sl_tables(self):
        """(nbr int32[n_tri, 4], trans float64[n_tri, 3, 2]) of the walk, internal order."""
        nbr = np.zeros((self.n_tri, 4), np.int32)
        trans = np.zeros((self.n_tri, 3, 2))
        _check(load().dgsl_query_sl_tables(self.h, C.c_void_p(nbr.ctypes.data), C.c_void_p(trans.ctypes.data)))
        return nbr, trans

    def node_coords(self, grid):
        n = self.n_dof if grid == MAIN else self.n_dual
        out = np.zeros((n, 2))
        _check(load().dgsl_node_coords(self.h, int(grid), C.c_void_p(out.ctypes.data)))
        return out

    def couplings(self):
        """(Kd [n_tri][n_phi][n_phi], Ko [n_tri][3][n_phi][n_phi], nbr [n_tri][3]),
        internal order (host_only or factored builds)."""
        n = self.n_phi
        Kd = np.zeros((self.n_tri, n, n))
        Ko = np.zeros((self.n_tri, 3, n, n))
        nbr = np.zeros((self.n_tri, 3), dtype=np.int32)
        _check(load().dgsl_query_couplings(self.h, C.c_void_p(Kd.ctypes.data), C.c_void_p(Ko.ctypes.data),
                                           C.c_void_p(nbr.ctypes.data)))
        return Kd, Ko, nbr

    def blocks(self):
        n, npsi = self.n_phi, self.n_psi
        G = np.zeros((self.n_edge, 2, 2, n, n))
        Minv = np.zeros((self.n_edge, npsi, npsi))
        Mref = np.zeros((n, n))
        area = np.zeros(self.n_tri)
        _check(load().dgsl_query_blocks(self.h, C.c_void_p(G.ctypes.data), C.c_void_p(Minv.ctypes.data),
                                        C.c_void_p(Mref.ctypes.data), C.c_void_p(area.ctypes.data)))
        return G, Minv, Mref, area

    # ---- device applies
    def dgsl_apply_schur(self, dt, x, y, n_rhs=1, form=FORM_ASSEMBLED, stream=None):
        n = self.n_dof * n_rhs
        _check(load().dgsl_apply_schur(self.h, int(form), float(dt), _dptr(x, "float64", n),
                                       _dptr(y, "float64", n), int(n_rhs), _stream(stream)))

    def dgsl_apply_schur_f32(self, dt, x, y, n_rhs=1, stream=None):
        n = self.n_dof * n_rhs
        _check(load().dgsl_apply_schur_f32(self.h, float(dt), _dptr(x, "float32", n),
                                           _dptr(y, "float32", n), int(n_rhs), _stream(stream)))

    def dgsl_apply_helmholtz(self, nu_dt, x, y, n_rhs=1, stream=None):
        n = self.n_dof * n_rhs
        _check(load().dgsl_apply_helmholtz(self.h, float(nu_dt), _dptr(x, "float64", n),
                                           _dptr(y, "float64", n), int(n_rhs), _stream(stream)))

    def dgsl_project_d2m_rhs(self, vhat, b, n_rhs=1, stream=None):
        _check(load().dgsl_project_d2m_rhs(self.h, _dptr(vhat, "float64", self.n_dual * n_rhs),
                                           _dptr(b, "float64", self.n_dof * n_rhs), int(n_rhs),
                                           _stream(stream)))

    def dgsl_project_m2d(self, vbar, vhat, n_rhs=1, stream=None):
        _check(load().dgsl_project_m2d(self.h, _dptr(vbar, "float64", self.n_dof * n_rhs),
                                       _dptr(vhat, "float64", self.n_dual * n_rhs), int(n_rhs),
                                       _stream(stream)))

    def dgsl_apply_div(self, vhat, y, n_rhs=1, stream=None):
        _check(load().dgsl_apply_div(self.h, _dptr(vhat, "float64", 2 * self.n_dual * n_rhs),
                                     _dptr(y, "float64", self.n_dof * n_rhs), int(n_rhs),
                                     _stream(stream)))

    def dgsl_velocity_update(self, coef, F, p, v, n_rhs=1, stream=None):
        """v = F - coef Mhat^-1 G p (eq. nc.2); F, v vector dual fields, p main fields."""
        _check(load().dgsl_velocity_update(self.h, float(coef), _dptr(F, "float64", 2 * self.n_dual * n_rhs),
                                           _dptr(p, "float64", self.n_dof * n_rhs),
                                           _dptr(v, "float64", 2 * self.n_dual * n_rhs), int(n_rhs),
                                           _stream(stream)))

    def dgsl_sl_transport(self, dt, vbar, c=None, cstar=None, n_fields=0, foot=None, cell=None, steps=None,
                          stream=None):
        """Semi-Lagrangian transport (Sec. 2.5, eq. intstage): vbar [2 * n_dof]
        float64; c, cstar [n_fields * n_dof] float64; optional foot
        [n_tri * n_g * 2] float64, cell and steps [n_tri * n_g] int32."""
        ng = sl_quadrature(self.p)[1].size
        nt = self.n_tri * ng
        opt = lambda t, dt_, m: _dptr(t, dt_, m) if t is not None else None  # noqa: E731
        _check(load().dgsl_sl_transport(
            self.h, float(dt), _dptr(vbar, "float64", 2 * self.n_dof),
            opt(c, "float64", n_fields * self.n_dof), opt(cstar, "float64", n_fields * self.n_dof), int(n_fields),
            opt(foot, "float64", 2 * nt), opt(cell, "int32", nt), opt(steps, "int32", nt), _stream(stream)))

    def dgsl_sl_transport_imex(self, R, dt, vbar, c=None, cstar=None, n_fields=0, foot=None, cell=None,
                               steps=None, stream=None):
        """Transport with the stage trajectories of the IMEX scheme of degree R
        (0, 1, 2); arguments as dgsl_sl_transport."""
        ng = sl_quadrature(self.p)[1].size
        nt = self.n_tri * ng
        opt = lambda t, dt_, m: _dptr(t, dt_, m) if t is not None else None  # noqa: E731
        _check(load().dgsl_sl_transport_imex(
            self.h, int(R), float(dt), _dptr(vbar, "float64", 2 * self.n_dof),
            opt(c, "float64", n_fields * self.n_dof), opt(cstar, "float64", n_fields * self.n_dof), int(n_fields),
            opt(foot, "float64", 2 * nt), opt(cell, "int32", nt), opt(steps, "int32", nt), _stream(stream)))

    def dgsl_ns_imex_step(self, R, dt, nu, vhat_in, vhat_out, p_out=None, opts=None, stream=None, check=True):
        """One SL-IMEX Navier-Stokes step (R = 0, 1, 2): vhat [2 * n_dual] float64
        (may alias), p_out [n_dof] or None.  Returns the dgsl_solve_info of the
        stage solves (per stage: Helmholtz x, Helmholtz y, Schur)."""
        if opts is None:
            opts = dgsl_default_solve_opts()
        ns = {0: 1, 1: 2, 2: 4}.get(int(R), 4)
        infos = (dgsl_solve_info * 12)()
        code = load().dgsl_ns_imex_step(self.h, int(R), float(dt), float(nu),
                                        _dptr(vhat_in, "float64", 2 * self.n_dual),
                                        _dptr(vhat_out, "float64", 2 * self.n_dual),
                                        _dptr(p_out, "float64", self.n_dof) if p_out is not None else None,
                                        C.byref(opts), infos, _stream(stream))
        if check:
            _check(code)
        return list(infos)[:3 * ns]

    def dgsl_advdiff_step(self, R, dt, alpha, vbar, c_in, c_out, opts=None, stream=None, check=True):
        """One SL-IMEX advection-diffusion step (R = 0, 1, 2): vbar [2 * n_dof],
        c_in, c_out [n_dof] float64 (may alias).  Returns the dgsl_solve_info of
        the stage solves (1, 2 or 4)."""
        if opts is None:
            opts = dgsl_default_solve_opts()
        ns = {0: 1, 1: 2, 2: 4}.get(int(R), 4)
        infos = (dgsl_solve_info * 4)()
        code = load().dgsl_advdiff_step(self.h, int(R), float(dt), float(alpha),
                                        _dptr(vbar, "float64", 2 * self.n_dof), _dptr(c_in, "float64", self.n_dof),
                                        _dptr(c_out, "float64", self.n_dof), C.byref(opts), infos, _stream(stream))
        if check:
            _check(code)
        return list(infos)[:ns]

    def dgsl_ns_step(self, dt, nu, vhat_in, vhat_out, p_out=None, opts=None, stream=None, check=True):
        """One first-order semi-Lagrangian Navier-Stokes step; vhat [2 * n_dual]
        float64 (may alias), p_out [n_dof] or None (with opts.use_x0 its
        contents start the pressure solve).  Returns the three
        dgsl_solve_info (Helmholtz x, Helmholtz y, Schur)."""
        if opts is None:
            opts = dgsl_default_solve_opts()
        infos = (dgsl_solve_info * 3)()
        code = load().dgsl_ns_step(self.h, float(dt), float(nu), _dptr(vhat_in, "float64", 2 * self.n_dual),
                                   _dptr(vhat_out, "float64", 2 * self.n_dual),
                                   _dptr(p_out, "float64", self.n_dof) if p_out is not None else None,
                                   C.byref(opts), infos, _stream(stream))
        if check:
            _check(code)
        return list(infos)

    def dgsl_cg_solve(self, kind, coef, b, x, n_rhs=1, opts=None, stream=None, check=True):
        """Returns a list of dgsl_solve_info (one per right-hand side)."""
        if opts is None:
            opts = dgsl_default_solve_opts()
        infos = (dgsl_solve_info * n_rhs)()
        n = self.n_dof * n_rhs
        code = load().dgsl_cg_solve(self.h, int(kind), float(coef), _dptr(b, "float64", n),
                                    _dptr(x, "float64", n), int(n_rhs), C.byref(opts), infos,
                                    _stream(stream))
        if check and code not in (OK,):
            _check(code)
        return list(infos)


def _noalloc_solve(self, kind, coef, b, x, n_rhs=1, opts=None, stream=None, check=True):
    """dgsl_cg_solve_noalloc: the solve with the library's fixed scratch array
    (no device allocation; operators up to 262,144 DOFs)."""
    if opts is None:
        opts = dgsl_default_solve_opts()
    infos = (dgsl_solve_info * n_rhs)()
    n = self.n_dof * n_rhs
    code = load().dgsl_cg_solve_noalloc(self.h, int(kind), float(coef), _dptr(b, "float64", n),
                                        _dptr(x, "float64", n), int(n_rhs), C.byref(opts), infos,
                                        _stream(stream))
    if check and code != OK:
        _check(code)
    return list(infos)


Operator.dgsl_cg_solve_noalloc = _noalloc_solve


def _apply_multigrid(self, kind, coef, r, z, precision=PREC_F32_IR, stream=None):
    """dgsl_apply_multigrid: z = M r once (float64 tensors for PREC_F64, else
    float32)."""
    dt = "float64" if precision == PREC_F64 else "float32"
    _check(load().dgsl_apply_multigrid(self.h, int(kind), float(coef), int(precision), _dptr(r, dt, self.n_dof),
                                       _dptr(z, dt, self.n_dof), _stream(stream)))


def _query_multigrid(self, kind, coef):
    """dgsl_query_multigrid: (level sizes, cvid [n_tri, 3] natural order,
    aggregates of every level but the last, as a list of arrays)."""
    info = dgsl_mg_info()
    _check(load().dgsl_query_multigrid(self.h, int(kind), float(coef), C.byref(info), None, None))
    sizes = [int(info.sizes[i]) for i in range(info.n_levels)]
    cvid = np.zeros((self.n_tri, 3), dtype=np.int32)
    agg = np.zeros(max(1, sum(sizes[:-1])), dtype=np.int32)
    _check(load().dgsl_query_multigrid(self.h, int(kind), float(coef), C.byref(info),
                                       cvid.ctypes.data_as(C.c_void_p), agg.ctypes.data_as(C.c_void_p)))
    out, o = [], 0
    for n in sizes[:-1]:
        out.append(agg[o:o + n].copy())
        o += n
    return sizes, cvid, out


Operator.dgsl_apply_multigrid = _apply_multigrid
Operator.dgsl_query_multigrid = _query_multigrid


def _set_fields(o, kw):
    names = {f for f, _ in type(o)._fields_}
    for k, v in kw.items():
        if k not in names:  # ctypes would add a plain attribute the library never sees
            raise TypeError(f"{type(o).__name__} has no field {k!r}")
        setattr(o, k, v)
    return o


def sl_quadrature(p):
    """(pts f64[n_g, 2], w f64[n_g]) of dgsl_sl_transport for degree p."""
    ng = C.c_int32()
    _check(load().dgsl_sl_quadrature(int(p), None, None, C.byref(ng)))
    pts = np.zeros((ng.value, 2))
    w = np.zeros(ng.value)
    _check(load().dgsl_sl_quadrature(int(p), C.c_void_p(pts.ctypes.data), C.c_void_p(w.ctypes.data), C.byref(ng)))
    return pts, w


def solve_opts(**kw):
    return _set_fields(dgsl_default_solve_opts(), kw)


def engine_opts(**kw):
    o = dgsl_engine_opts()
    load().dgsl_default_engine_opts(C.byref(o))
    return _set_fields(o, kw)


def request(op, kind, coef, b, x, tol=0.0, n_rhs=1):
    """dgsl_request for device tensors b, x (float64, n_rhs * op.n_dof elements).
    The request holds raw device pointers: keep b and x alive until it completes."""
    if not 1 <= int(n_rhs) <= MAX_RHS:
        raise DgslError(EINVAL, f"n_rhs must be 1..{MAX_RHS}")
    m = int(n_rhs) * op.n_dof
    return dgsl_request(op.h.value, int(kind), int(n_rhs), float(coef), _dptr(b, "float64", m).value,
                        _dptr(x, "float64", m).value, float(tol))


def dgsl_cg_solve_batch(reqs, opts=None, stream=None, check=False):
    """Runs the requests in one persistent launch; returns their solve infos."""
    n = len(reqs)
    arr = (dgsl_request * n)(*reqs)
    infos = (dgsl_solve_info * n)()
    o = opts if opts is not None else engine_opts()
    code = load().dgsl_cg_solve_batch(arr, n, C.byref(o), infos, _stream(stream))
    if check:
        _check(code)
    elif code not in (OK, ENOTCONV, ETIMEOUT):
        _check(code)
    return list(infos)


class Server:
    """Request loop with continuous batching (dgsl_server_*)."""

    def __init__(self, opts=None):
        o = opts if opts is not None else engine_opts()
        h = C.c_void_p()
        _check(load().dgsl_server_create(C.byref(o), C.byref(h)))
        self.h = h

    def dgsl_submit(self, req):
        t = C.c_uint64()
        _check(load().dgsl_submit(self.h, C.byref(req), C.byref(t)))
        return t.value

    def dgsl_poll(self, ticket):
        """None while pending, else the request's dgsl_solve_info."""
        info = dgsl_solve_info()
        code = load().dgsl_poll(self.h, C.c_uint64(ticket), C.byref(info))
        if code == EPENDING:
            return None
        _check(code)
        return info

    def dgsl_poll_many(self, tickets):
        """tickets: numpy uint64 array -> (done int32 array, infos array)."""
        n = len(tickets)
        tk = np.ascontiguousarray(tickets, dtype=np.uint64)
        done = np.zeros(n, dtype=np.int32)
        infos = (dgsl_solve_info * max(n, 1))()
        code = load().dgsl_poll_many(self.h, C.c_void_p(tk.ctypes.data), n, C.cast(infos, C.c_void_p),
                                     C.c_void_p(done.ctypes.data))
        if code < 0:
            _check(-code)
        return done, infos

    def dgsl_cancel(self, ticket):
        code = load().dgsl_cancel(self.h, C.c_uint64(ticket))
        if code not in (OK, EPENDING):
            _check(code)
        return code == OK

    def stats(self):
        s = dgsl_server_stats()
        _check(load().dgsl_server_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in dgsl_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().dgsl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgsl_measure_fma_rate(fp64=True, device=0):
    """Measured FMA throughput of the device in flop/s (2 per FMA)."""
    v = C.c_double(0.0)
    _check(load().dgsl_measure_fma_rate(int(device), int(bool(fp64)), C.byref(v)))
    return v.value


def dgsl_selftest_wait_timeout(which, timeout_s=0.2, device=0):
    """Status (ETIMEOUT expected) of a bounded wait made to run out."""
    st = C.c_int(-1)
    _check(load().dgsl_selftest_wait_timeout(int(device), int(which), float(timeout_s), C.byref(st)))
    return st.value
