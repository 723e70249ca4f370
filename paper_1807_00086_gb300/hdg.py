"""Python binding of libhdg.so (ctypes). Argument marshalling only: every step of the
hot path runs in the library's CUDA kernels. Torch tensors are used as device buffers
(contiguous float64 on the context's device); the context is bound to the torch stream
that is current when it is created.

Names follow include/hdg.h: hdg_setup, hdg_condense, hdg_trace_apply, hdg_condensed_rhs,
hdg_trace_solve, hdg_recover, hdg_step, ...
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdg.so")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_double, P_int32 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)

HDG_BE, HDG_BDF2, HDG_DIRK3 = 1, 2, 3
HDG_FP64, HDG_MIXED, HDG_MIXED16 = 0, 1, 2
SCHEMES = {"be": HDG_BE, "bdf2": HDG_BDF2, "dirk3": HDG_DIRK3}
STATUS = {0: "HDG_OK", -1: "HDG_EINVAL", -2: "HDG_ENOMEM", -3: "HDG_ECUDA", -4: "HDG_ENOCONV",
          -5: "HDG_ETIMEOUT", -6: "HDG_ESTATE"}


class Mesh(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("n_vert", c_int64), ("n_elem", c_int64), ("vert", P_double),
                ("elem_vert", P_int32), ("elem_k", P_int32)]


class Material(ctypes.Structure):
    _fields_ = [("phys", c_int32), ("rho", P_double), ("c", P_double), ("lam", P_double), ("mu", P_double)]


class Options(ctypes.Structure):
    _fields_ = [("prec", c_int32), ("rtol", c_double), ("maxit", c_int32), ("check_every", c_int32),
                ("inner_rtol", c_double), ("max_sweeps", c_int32), ("nrhs", c_int32), ("use_graphs", c_int32),
                ("guess_history", c_int32), ("device_loops", c_int32), ("trace_space", c_int32),
                ("solver", c_int32), ("gmres_restart", c_int32), ("newton_tol", c_double), ("newton_maxit", c_int32),
                ("precond", c_int32)]


class Sizes(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("k", c_int32), ("Np", c_int32), ("Nf", c_int32), ("n_local", c_int32),
                ("n_trace_local", c_int32), ("n_elem", c_int64), ("n_faces", c_int64), ("n_bnd_faces", c_int64),
                ("nq_vol", c_int32), ("nq_face", c_int32), ("device_bytes", c_int64), ("field_entries", c_int64),
                ("trace_entries", c_int64), ("schur_entries", c_int64), ("slot_entries", c_int64),
                ("trace_unknowns", c_int64)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("sweeps", c_int32), ("rel_residual", c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "sweeps": self.sweeps, "rel_residual": self.rel_residual}


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", c_int64), ("apply_launches", c_int64), ("apply_ms", c_double),
                ("apply32_launches", c_int64), ("apply32_ms", c_double), ("applydf_launches", c_int64),
                ("applydf_ms", c_double), ("apply16_launches", c_int64), ("apply16_ms", c_double),
                ("dev_apply32_launches", c_int64), ("dev_apply32_ms", c_double),
                ("dev_apply16_launches", c_int64), ("dev_apply16_ms", c_double),
                ("svk_condense_launches", c_int64), ("svk_condense_ms", c_double),
                ("svk_recover_launches", c_int64), ("svk_recover_ms", c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("tuned", c_int32), ("apply32_warps", c_int32), ("apply32_unroll", c_int32),
                ("apply64_warps", c_int32), ("apply64_unroll", c_int32), ("local_threads", c_int32 * 2)]


# hdg_svk_forcing: int32 (*)(void* user, double t, double* f_host, double* g_host)
FORCING = ctypes.CFUNCTYPE(c_int32, c_void_p, c_double, ctypes.POINTER(c_double), ctypes.POINTER(c_double))


# exported entry points: name -> (restype, argtypes)
SIGNATURES = {
    "hdg_default_options": (None, [ctypes.POINTER(Options)]),
    "hdg_setup": (c_int32, [ctypes.POINTER(Mesh), c_int32, c_double, ctypes.POINTER(Material),
                            ctypes.POINTER(Options), c_void_p, ctypes.POINTER(c_void_p)]),
    "hdg_destroy": (None, [c_void_p]),
    "hdg_last_error": (ctypes.c_char_p, [c_void_p]),
    "hdg_get_sizes": (c_int32, [c_void_p, ctypes.POINTER(Sizes)]),
    "hdg_condense": (c_int32, [c_void_p, c_double]),
    "hdg_get_schur": (c_int32, [c_void_p, c_void_p]),
    "hdg_trace_apply": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "hdg_condensed_rhs": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hdg_trace_solve": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(SolveInfo)]),
    "hdg_recover": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hdg_postprocess": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hdg_host_skeleton": (c_int32, [c_int32, c_int64, c_int64, P_double, P_int32, ctypes.POINTER(c_int64), P_int32,
                                    P_int32, P_int32, P_double]),
    "hdg_host_tables": (c_int32, [c_int32, c_int32, P_double, P_double, P_double, P_double]),
    "hdg_host_trace_nodes": (c_int32, [c_int32, c_int64, c_int64, P_double, P_int32, c_int32, c_int32,
                                       ctypes.POINTER(c_int64), P_int32, P_double]),
    "hdg_set_sources": (c_int32, [c_void_p, c_int32, P_double, P_double, P_int32, P_double, c_double, c_double]),
    "hdg_reset_column": (c_int32, [c_void_p, c_int32]),
    "hdg_stream_create": (c_int32, [ctypes.POINTER(c_void_p)]),
    "hdg_stream_destroy": (c_int32, [c_void_p]),
    "hdg_set_stream": (c_int32, [c_void_p, c_void_p]),
    "hdg_precond_apply": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "hdg_svk_set_traction_faces": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_uint8)]),
    "hdg_svk_set_forcing": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "hdg_svk_newton_counts": (c_int32, [c_void_p, P_int32, c_int32, P_int32]),
    "hdg_quadrature_points": (c_int32, [c_void_p, c_int32, P_double]),
    "hdg_project_volume": (c_int32, [c_void_p, P_double, c_void_p]),
    "hdg_set_dirichlet": (c_int32, [c_void_p, P_double, c_double, c_double]),
    "hdg_set_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_double]),
    "hdg_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "hdg_step": (c_int32, [c_void_p, c_double, c_int32, c_int32, ctypes.POINTER(SolveInfo)]),
    "hdg_checkpoint_size": (c_int32, [c_void_p, ctypes.POINTER(c_int64)]),
    "hdg_save_checkpoint": (c_int32, [c_void_p, c_void_p]),
    "hdg_load_checkpoint": (c_int32, [c_void_p, c_void_p]),
    "hdg_trace_apply_noalloc": (c_int32, [c_int32, c_int32, c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, ctypes.c_char_p, c_int32]),
    "hdg_enable_stats": (c_int32, [c_void_p, c_int32]),
    "hdg_get_stats": (c_int32, [c_void_p, ctypes.POINTER(Stats), c_int32]),
    "hdg_get_tuning": (c_int32, [c_void_p, ctypes.POINTER(Tuning)]),
}

_lib = None


def load():
    """Load libhdg.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhdg.so is not built (run __graft_entry__.build()); no CPU fallback exists")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def own_stream():
    """A dedicated CUDA stream created by the library (torch.cuda.ExternalStream wrapper).
    torch.cuda.Stream() draws from a small per-device pool, so many contexts would share
    streams; the caller must call release_stream() after closing the context."""
    import torch
    lib = load()
    p = ctypes.c_void_p()
    st = lib.hdg_stream_create(ctypes.byref(p))
    if st != 0:
        raise HDGError(st, "hdg_stream_create failed")
    return torch.cuda.ExternalStream(p.value)


def release_stream(stream):
    load().hdg_stream_destroy(ctypes.c_void_p(stream.cuda_stream))


class HDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _np_ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Solver:
    """One HDG problem resident on the current CUDA device (wraps an hdg_ctx)."""

    def __init__(self, vert, elem, k, tau, rho, c=None, prec="fp64", rtol=1e-13, maxit=2000, check_every=16,
                 inner_rtol=None, max_sweeps=None, nrhs=1, use_graphs=False, stream=None, lam=None, mu=None,
                 elem_k=None, guess_history=None, device_loops=None, trace_space="hdg", solver="cg",
                 gmres_restart=None, svk=False, newton_tol=None, newton_maxit=None, precond="jacobi"):
        """Acoustic when `c` is given (rho, c); elastic when `lam` and `mu` are given (rho, lam, mu);
        svk=True with lam, mu: nonlinear Saint Venant-Kirchhoff elastodynamics (Newton per stage).
        elem_k: per-element degrees (3D elastic); fields and traces are then flat vectors.
        trace_space: "hdg", "iedg" or "edg" (continuous traces on the interior / all faces).
        solver: "cg" (default) or "gmres" (restarted GMRES with two-pass classical Gram-Schmidt).
        precond: the GMRES right preconditioner, "jacobi" (default) or "bilu0" (block ILU(0))."""
        import torch
        self.lib = load()
        self.torch = torch
        vert = np.ascontiguousarray(vert, dtype=np.float64)
        elem = np.ascontiguousarray(elem, dtype=np.int32)
        ne = elem.shape[0]
        arr = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ne,)))
        self._rho = arr(rho)
        self.elastic = lam is not None
        if self.elastic:
            self._lam, self._mu = arr(lam), arr(mu)
            self._c = arr(1.0)
            mat = Material(2 if svk else 1, _np_ptr(self._rho, c_double), _np_ptr(self._c, c_double),
                           _np_ptr(self._lam, c_double), _np_ptr(self._mu, c_double))
        else:
            self._c = arr(c)
            mat = Material(0, _np_ptr(self._rho, c_double), _np_ptr(self._c, c_double), None, None)
        self._ek = None if elem_k is None else np.ascontiguousarray(elem_k, dtype=np.int32)
        mesh = Mesh(vert.shape[1], vert.shape[0], ne, _np_ptr(vert, c_double), _np_ptr(elem, c_int32),
                    None if self._ek is None else _np_ptr(self._ek, c_int32))
        opt = Options()
        self.lib.hdg_default_options(ctypes.byref(opt))
        opt.prec = {"fp64": HDG_FP64, "mixed": HDG_MIXED, "mixed16": HDG_MIXED16}[prec]
        opt.rtol, opt.maxit, opt.check_every = rtol, maxit, check_every
        if inner_rtol is not None:
            opt.inner_rtol = inner_rtol
        if max_sweeps is not None:
            opt.max_sweeps = max_sweeps
        opt.nrhs = nrhs
        opt.use_graphs = 1 if use_graphs else 0
        if guess_history is not None:
            opt.guess_history = guess_history
        if device_loops is not None:
            opt.device_loops = 1 if device_loops else 0
        opt.trace_space = {"hdg": 0, "iedg": 1, "edg": 2}[trace_space]
        opt.solver = {"cg": 0, "gmres": 1}[solver]
        if gmres_restart is not None:
            opt.gmres_restart = gmres_restart
        opt.precond = {"jacobi": 0, "bilu0": 1}[precond]
        if newton_tol is not None:
            opt.newton_tol = newton_tol
        if newton_maxit is not None:
            opt.newton_maxit = newton_maxit
        self.svk = bool(svk)
        self._forcing_cb = None
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = self.lib.hdg_setup(ctypes.byref(mesh), k, tau, ctypes.byref(mat), ctypes.byref(opt),
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ctx))
        self.ctx = ctx
        self._check(st)
        sz = Sizes()
        self._check(self.lib.hdg_get_sizes(self.ctx, ctypes.byref(sz)))
        self.sizes = sz
        self.dim, self.k, self.Np, self.Nf = sz.dim, sz.k, sz.Np, sz.Nf
        self.n, self.m = sz.n_local, sz.n_trace_local
        self.n_elem, self.n_faces, self.n_bnd = sz.n_elem, sz.n_faces, sz.n_bnd_faces
        self.R = nrhs
        self.vardeg = self.n == 0
        if self.vardeg:
            self._fshape, self._tshape = (sz.field_entries,), (sz.trace_entries,)
        else:
            self._fshape = (self.n_elem, self.n) if nrhs == 1 else (self.n_elem, self.n, nrhs)
            self._tshape = (self.n_faces, self.Nf) if nrhs == 1 else (self.n_faces, self.Nf, nrhs)

    def _check(self, st):
        if st != 0:
            msg = self.lib.hdg_last_error(self.ctx)
            raise HDGError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.hdg_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # buffers -------------------------------------------------------------------------------
    def empty_fields(self):
        return self.torch.zeros(self._fshape, dtype=self.torch.float64, device=self.device)

    def empty_traces(self):
        return self.torch.zeros(self._tshape, dtype=self.torch.float64, device=self.device)

    def _dev(self, t, shape):
        assert t.dtype == self.torch.float64 and t.is_cuda and t.is_contiguous(), "float64 contiguous CUDA tensor"
        assert t.numel() == int(np.prod(shape)), (tuple(t.shape), shape)
        return _ptr(t)

    # entry points --------------------------------------------------------------------------
    def hdg_set_stream(self, stream):
        """Rebind the context to `stream` (a torch.cuda.Stream or ExternalStream)."""
        self._check(self.lib.hdg_set_stream(self.ctx, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def hdg_precond_apply(self, r, z=None):
        """z = M^{-1} r with the GMRES preconditioner (Jacobi or block ILU(0)) for sgn K."""
        z = self.empty_traces() if z is None else z
        self._check(self.lib.hdg_precond_apply(self.ctx, self._dev(r, self._tshape), self._dev(z, self._tshape)))
        return z

    # nonlinear elastodynamics ---------------------------------------------------------------
    def hdg_svk_set_traction_faces(self, mask):
        """mask [n_bnd] (order of hdg_quadrature_points(1)): 1 = traction face, None clears."""
        if mask is None:
            self._check(self.lib.hdg_svk_set_traction_faces(self.ctx, None))
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        assert m.shape == (self.n_bnd,)
        self._check(self.lib.hdg_svk_set_traction_faces(self.ctx, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def hdg_svk_set_forcing(self, fn):
        """fn(t, f, g) fills f [n_elem, nq_vol, 3] (body force at the volume points) and
        g [n_bnd, nq_face, 3] (traction P n at the boundary-face points) in place; None removes it."""
        if fn is None:
            self._forcing_cb = None
            self._check(self.lib.hdg_svk_set_forcing(self.ctx, None, None))
            return
        sz = self.sizes
        fshape = (self.n_elem, sz.nq_vol, 3)
        gshape = (max(self.n_bnd, 1), sz.nq_face, 3)

        def cb(user, t, fptr, gptr):
            try:
                f = np.ctypeslib.as_array(fptr, shape=fshape)
                g = np.ctypeslib.as_array(gptr, shape=gshape)
                fn(t, f, g[:self.n_bnd])
                return 0
            except Exception:   # reported to the library as a failed callback
                return 1
        self._forcing_cb = FORCING(cb)
        self._check(self.lib.hdg_svk_set_forcing(self.ctx, ctypes.cast(self._forcing_cb, c_void_p), None))

    def hdg_svk_newton_counts(self):
        n = c_int32()
        self._check(self.lib.hdg_svk_newton_counts(self.ctx, None, 0, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        self._check(self.lib.hdg_svk_newton_counts(self.ctx, _np_ptr(out, c_int32), n.value, ctypes.byref(n)))
        return out[:n.value].tolist()

    def hdg_condense(self, alpha):
        self._check(self.lib.hdg_condense(self.ctx, alpha))

    def hdg_get_schur(self):
        S = self.torch.empty((self.n_elem, self.m, self.m), dtype=self.torch.float64, device=self.device)
        self._check(self.lib.hdg_get_schur(self.ctx, _ptr(S)))
        return S

    def hdg_trace_apply(self, x, y=None):
        y = self.empty_traces() if y is None else y
        self._check(self.lib.hdg_trace_apply(self.ctx, self._dev(x, self._tshape),
                                             self._dev(y, self._tshape)))
        return y

    def hdg_condensed_rhs(self, F, lamD=None, r=None):
        r = self.empty_traces() if r is None else r
        self._check(self.lib.hdg_condensed_rhs(self.ctx, self._dev(F, self._fshape),
                                               None if lamD is None else self._dev(lamD, self._tshape),
                                               self._dev(r, self._tshape)))
        return r

    def hdg_trace_solve(self, r, lam):
        info = SolveInfo()
        self._check(self.lib.hdg_trace_solve(self.ctx, self._dev(r, self._tshape),
                                             self._dev(lam, self._tshape), ctypes.byref(info)))
        return info.as_dict()

    def hdg_recover(self, F, lam, u=None):
        u = self.empty_fields() if u is None else u
        self._check(self.lib.hdg_recover(self.ctx, self._dev(F, self._fshape),
                                         self._dev(lam, self._tshape), self._dev(u, self._fshape)))
        return u

    def hdg_postprocess(self, u, lam, pstar=None):
        """Post-processed pressure p* in P_{k+1} per element, [n_elem, Np(k+1)]."""
        np1 = math.comb(self.k + 1 + self.dim, self.dim)
        if pstar is None:
            pstar = self.torch.zeros((self.n_elem, np1), dtype=self.torch.float64, device=self.device)
        self._check(self.lib.hdg_postprocess(self.ctx, self._dev(u, self._fshape), self._dev(lam, self._tshape),
                                             self._dev(pstar, (self.n_elem, np1))))
        return pstar

    def hdg_set_sources(self, pos, amp, f0, t0, col=None, delay=None):
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, self.dim))
        amp = np.ascontiguousarray(np.broadcast_to(np.asarray(amp, dtype=np.float64), (pos.shape[0],)))
        colp = None
        if col is not None:
            col = np.ascontiguousarray(np.asarray(col, dtype=np.int32).reshape(-1))
            colp = _np_ptr(col, c_int32)
        delp = None
        if delay is not None:
            delay = np.ascontiguousarray(np.asarray(delay, dtype=np.float64).reshape(-1))
            delp = _np_ptr(delay, c_double)
        self._check(self.lib.hdg_set_sources(self.ctx, pos.shape[0], _np_ptr(pos, c_double), _np_ptr(amp, c_double),
                                             colp, delp, f0, t0))

    def hdg_reset_column(self, j):
        self._check(self.lib.hdg_reset_column(self.ctx, j))

    def vol_points_per_element(self):
        """Volume quadrature points of each element ((k_K + 2)^dim with per-element degrees)."""
        if self.vardeg:
            return (self._ek.astype(np.int64) + 2) ** self.dim if self._ek is not None else \
                np.full(self.n_elem, (self.k + 2) ** self.dim)
        return np.full(self.n_elem, self.sizes.nq_vol)

    def hdg_quadrature_points(self, which):
        if self.vardeg and which == 0:
            out = np.zeros((int(self.vol_points_per_element().sum()), self.dim))
            self._check(self.lib.hdg_quadrature_points(self.ctx, which, _np_ptr(out, c_double)))
            return out
        nq = self.sizes.nq_vol if which == 0 else self.sizes.nq_face
        cnt = self.n_elem if which == 0 else self.n_bnd
        out = np.zeros((cnt, nq, self.dim))
        self._check(self.lib.hdg_quadrature_points(self.ctx, which, _np_ptr(out, c_double)))
        return out

    def hdg_project_volume(self, vals, u=None):
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        ncomp = 21 if self.svk else (self.dim + self.dim * (self.dim + 1) // 2) if self.elastic else self.dim + 1
        if self.vardeg:
            assert vals.shape == (int(self.vol_points_per_element().sum()), ncomp)
        else:
            assert vals.shape == (self.n_elem, self.sizes.nq_vol, ncomp)
        u = self.empty_fields() if u is None else u
        self._check(self.lib.hdg_project_volume(self.ctx, _np_ptr(vals, c_double), self._dev(u, self._fshape)))
        return u

    def hdg_set_dirichlet(self, vals=None, omega=0.0, phase=0.0):
        if vals is None:
            self._check(self.lib.hdg_set_dirichlet(self.ctx, None, omega, phase))
            return
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        assert vals.shape == (self.n_bnd, self.sizes.nq_face)
        self._check(self.lib.hdg_set_dirichlet(self.ctx, _np_ptr(vals, c_double), omega, phase))

    def _state(self, t, shape):
        """a CUDA tensor or a page-locked CPU tensor (the state calls copy either way)"""
        if not t.is_cuda:
            assert t.dtype == self.torch.float64 and t.is_contiguous() and t.is_pinned(), "pinned float64 CPU tensor"
            assert t.numel() == int(np.prod(shape)), (tuple(t.shape), shape)
            return _ptr(t)
        return self._dev(t, shape)

    def hdg_set_state(self, u, t=0.0, uprev=None, lam=None):
        """u, uprev, lam: CUDA tensors or page-locked CPU tensors."""
        shp = self._fshape
        self._check(self.lib.hdg_set_state(self.ctx, self._state(u, shp),
                                           None if uprev is None else self._state(uprev, shp),
                                           None if lam is None else self._state(lam, self._tshape), t))

    def hdg_get_state(self, u=None, uprev=None, lam=None, want_prev=False):
        """Returns (u, lam, t) or, with want_prev, (u, uprev, lam, t); buffers may be passed in."""
        u = self.empty_fields() if u is None else u
        lam = self.empty_traces() if lam is None else lam
        if want_prev and uprev is None:
            uprev = self.empty_fields()
        t = ctypes.c_double()
        self._check(self.lib.hdg_get_state(self.ctx, self._state(u, self._fshape),
                                           self._state(uprev, self._fshape) if uprev is not None else None,
                                           self._state(lam, self._tshape), ctypes.byref(t)))
        return (u, uprev, lam, t.value) if want_prev else (u, lam, t.value)

    def hdg_enable_stats(self, enable=True):
        self._check(self.lib.hdg_enable_stats(self.ctx, 1 if enable else 0))

    def hdg_get_stats(self, reset=False):
        st = Stats()
        self._check(self.lib.hdg_get_stats(self.ctx, ctypes.byref(st), 1 if reset else 0))
        return {"kernel_launches": st.kernel_launches, "apply_launches": st.apply_launches, "apply_ms": st.apply_ms,
                "apply32_launches": st.apply32_launches, "apply32_ms": st.apply32_ms,
                "applydf_launches": st.applydf_launches, "applydf_ms": st.applydf_ms,
                "apply16_launches": st.apply16_launches, "apply16_ms": st.apply16_ms,
                "dev_apply32_launches": st.dev_apply32_launches, "dev_apply32_ms": st.dev_apply32_ms,
                "dev_apply16_launches": st.dev_apply16_launches, "dev_apply16_ms": st.dev_apply16_ms,
                "svk_condense_launches": st.svk_condense_launches, "svk_condense_ms": st.svk_condense_ms,
                "svk_recover_launches": st.svk_recover_launches, "svk_recover_ms": st.svk_recover_ms}

    def hdg_get_tuning(self):
        """Autotuned tiles of a per-element-degree context (see hdg_tuning in include/hdg.h)."""
        t = Tuning()
        self._check(self.lib.hdg_get_tuning(self.ctx, ctypes.byref(t)))
        return {"tuned": t.tuned, "apply32_tile": (t.apply32_warps, t.apply32_unroll),
                "apply64_tile": (t.apply64_warps, t.apply64_unroll), "local_threads": tuple(t.local_threads)}

    def hdg_save_checkpoint(self):
        """The complete solver state as a host byte array (bitwise resume with hdg_load_checkpoint)."""
        n = c_int64()
        self._check(self.lib.hdg_checkpoint_size(self.ctx, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        self._check(self.lib.hdg_save_checkpoint(self.ctx, buf.ctypes.data_as(c_void_p)))
        return buf

    def hdg_load_checkpoint(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.hdg_load_checkpoint(self.ctx, buf.ctypes.data_as(c_void_p)))

    def hdg_step(self, dt, scheme, nsteps=1):
        info = SolveInfo()
        self._check(self.lib.hdg_step(self.ctx, dt, SCHEMES[scheme] if isinstance(scheme, str) else scheme, nsteps,
                                      ctypes.byref(info)))
        return info.as_dict()
