"""Python binding of the GB300 radiative-transfer library (C ABI in include/rt.h).

Argument marshalling only: every step of assembly, apply and solve runs in the
CUDA library ``librt.so``.  Device arrays are passed as torch tensors (their
data pointers) together with the CUDA stream to run on.  Every call goes
through :func:`lib`, which raises ImportError when the library has not been
built -- there is no CPU fallback.

Names follow the C ABI: :func:`rt_build_operator`, :meth:`Operator.apply`
(``rt_apply``), :meth:`Operator.source` (``rt_source``),
:meth:`Operator.eval_entries` (``rt_eval_entries``),
:meth:`Operator.solve_fixed_point` (``rt_solve_fixed_point``),
:meth:`Operator.info` (``rt_operator_info``), :func:`rt_plan`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOCONV, RT_ETIMEOUT, RT_EAGAIN = 0, -1, -2, -3, -4, -5, -6
RT_KAPPA_CONST, RT_KAPPA_SINPROD, RT_KAPPA_GRID = 0, 1, 2
RT_MODE_DENSE, RT_MODE_HMATRIX = 0, 1
RT_PREC_F64, RT_PREC_F32, RT_PREC_BF16, RT_PREC_F16 = 0, 1, 2, 3
RT_ADM_GAP, RT_ADM_CENTER = 0, 1
RT_LINE_CLOSED, RT_LINE_NODES = 0, 1

_c_i64 = ctypes.c_int64
_c_int = ctypes.c_int
_c_dbl = ctypes.c_double
_P = ctypes.c_void_p


class RtMesh(ctypes.Structure):
    _fields_ = [("n_vert", _c_i64), ("xyz", _P), ("n_tet", _c_i64), ("tet", _P)]


class RtKappa(ctypes.Structure):
    _fields_ = [("kind", _c_int), ("k0", _c_dbl), ("amp", _c_dbl), ("grid", _P), ("dims", _c_int * 3),
                ("bbox", _c_dbl * 6)]


class RtBox(ctypes.Structure):
    _fields_ = [("lo", _c_dbl * 3), ("hi", _c_dbl * 3)]


class RtWall(ctypes.Structure):
    _fields_ = [("p", _c_dbl * 3), ("n", _c_dbl * 3), ("R0", _c_dbl)]


class RtFreqs(ctypes.Structure):
    _fields_ = [("F", _c_int), ("nu", _P), ("w", _P), ("c", _P), ("albedo", _P), ("group", _P)]


class RtProblem(ctypes.Structure):
    _fields_ = [("mesh", RtMesh), ("kappa", RtKappa), ("n_walls", _c_int), ("walls", _P), ("n_emit", _c_i64),
                ("emit_tri", _P), ("Q0", _c_dbl), ("T_emit", _c_dbl), ("grey", _c_int), ("freqs", RtFreqs),
                ("corner", _c_int), ("n_obstacles", _c_int), ("obstacles", _P)]


class RtHparams(ctypes.Structure):
    _fields_ = [("mode", _c_int), ("prec", _c_int), ("far_prec", _c_int), ("aca_eps", _c_dbl), ("leaf", _c_int),
                ("eta", _c_dbl), ("gauss_pts", _c_int), ("rank_max", _c_int), ("adm", _c_int),
                ("line_eval", _c_int), ("refine", _c_int), ("tensor_cores", _c_int), ("wave_bytes", _c_i64),
                ("kappa_bins", _c_int)]


class RtInfo(ctypes.Structure):
    _fields_ = [("N", _c_i64), ("F", _c_i64), ("G", _c_i64), ("mode", _c_int), ("prec", _c_int), ("far_prec", _c_int),
                ("n_leaves", _c_i64), ("n_near", _c_i64), ("n_far", _c_i64), ("n_dense_fallback", _c_i64),
                ("stored_entries", _c_i64), ("compression", _c_dbl), ("rank_min", _c_i64), ("rank_max", _c_i64),
                ("rank_sum", _c_i64), ("aca_steps", _c_i64), ("entries_evaluated", _c_i64),
                ("apply_bytes", _c_i64), ("apply_flops", _c_i64), ("device_bytes", _c_i64),
                ("ms_tree", _c_dbl), ("ms_near", _c_dbl), ("ms_aca", _c_dbl), ("ms_pack", _c_dbl),
                ("ms_source", _c_dbl), ("peak_bytes", _c_i64), ("aca_waves", _c_i64),
                ("apply_tensor_cores", _c_i64), ("assembly_terms", _c_i64), ("assembly_depths", _c_i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RtSourceInfo(ctypes.Structure):
    _fields_ = [("N", _c_i64), ("L", _c_i64), ("G", _c_i64), ("n_blocks", _c_i64), ("n_far", _c_i64),
                ("n_dense", _c_i64), ("rank_sum", _c_i64), ("rank_max", _c_i64), ("stored_entries", _c_i64),
                ("compression", _c_dbl), ("apply_bytes", _c_i64), ("device_bytes", _c_i64), ("ms_eval", _c_dbl),
                ("ms_aca", _c_dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RtSolveOpts(ctypes.Structure):
    _fields_ = [("tol", _c_dbl), ("max_iter", _c_int), ("check_every", _c_int), ("T0", _c_dbl), ("use_J0", _c_int),
                ("use_graph", _c_int), ("refine_tol", _c_dbl)]


class RtBatchInfo(ctypes.Structure):
    _fields_ = [("count", _c_i64), ("total_vec", _c_i64), ("total_vert", _c_i64), ("p1_target_bytes", _c_int),
                ("ctas_per_sm", _c_int), ("n_works", _c_int), ("apply_bytes", _c_i64), ("tune_ms", _c_dbl),
                ("build_ms", _c_dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RtServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", _c_i64), ("slots", _c_int), ("max_bypass", _c_int), ("hp", RtHparams),
                ("opts", RtSolveOpts)]


class RtRequestInfo(ctypes.Structure):
    _fields_ = [("status", _c_int), ("iters", _c_int), ("converged", _c_int), ("residual", _c_dbl), ("N", _c_i64),
                ("F", _c_i64), ("est_bytes", _c_i64), ("peak_bytes", _c_i64), ("resident_bytes", _c_i64),
                ("t_submit", _c_dbl), ("t_admit", _c_dbl), ("t_built", _c_dbl), ("t_done", _c_dbl),
                ("ms_build", _c_dbl), ("ms_solve", _c_dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RtServerInfo(ctypes.Structure):
    _fields_ = [("submitted", _c_i64), ("finished", _c_i64), ("failed", _c_i64), ("queued", _c_i64),
                ("running", _c_i64), ("reserved_bytes", _c_i64), ("peak_reserved_bytes", _c_i64),
                ("max_running", _c_i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RtSolveStats(ctypes.Structure):
    _fields_ = [("iters", _c_int), ("converged", _c_int), ("residual", _c_dbl), ("ms_total", _c_dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol declared in include/rt.h
EXPORTS = ("rt_build_operator", "rt_operator_info", "rt_apply", "rt_apply_group", "rt_apply_noalloc", "rt_source", "rt_eval_entries",
           "rt_build_source_operator", "rt_source_operator_info", "rt_apply_source", "rt_source_free",
           "rt_eval_sin2pi", "rt_solve_fixed_point", "rt_free", "rt_last_error", "rt_plan", "rt_build_batch",
           "rt_batch_info", "rt_batch_apply", "rt_solve_batch", "rt_batch_set_wait", "rt_batch_free",
           "rt_batch_last_error", "rt_server_create", "rt_submit", "rt_poll", "rt_server_info", "rt_server_free")

_lib = None


def lib():
    """Load librt.so (built by ``paper_2306_05789_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2306_05789_gb300.build` "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.rt_build_operator.argtypes = [ctypes.POINTER(RtProblem), ctypes.POINTER(RtHparams), _P, ctypes.POINTER(_P)]
    L.rt_operator_info.argtypes = [_P, ctypes.POINTER(RtInfo)]
    L.rt_apply.argtypes = [_P, _P, _P, _P]
    L.rt_apply_noalloc.argtypes = [_P, _P, _P, _P]
    L.rt_apply_group.argtypes = [_P, _c_int, _P, _c_i64, _c_int, _P, _c_i64, _P]
    L.rt_source.argtypes = [_P, _P, _P]
    L.rt_eval_entries.argtypes = [_P, _c_int, _c_i64, _P, _P, _P, _P]
    L.rt_eval_sin2pi.argtypes = [_P, _P, _P, _c_i64, _P]
    L.rt_build_source_operator.argtypes = [_P, _P, ctypes.POINTER(_P)]
    L.rt_source_operator_info.argtypes = [_P, ctypes.POINTER(RtSourceInfo), _P]
    L.rt_apply_source.argtypes = [_P, _P, _P, _P]
    L.rt_source_free.argtypes = [_P]
    L.rt_source_free.restype = None
    L.rt_solve_fixed_point.argtypes = [_P, ctypes.POINTER(RtSolveOpts), _P, _P, ctypes.POINTER(RtSolveStats), _P]
    L.rt_free.argtypes = [_P]
    L.rt_free.restype = None
    L.rt_last_error.restype = ctypes.c_char_p
    L.rt_plan.argtypes = [_P, _c_i64, _c_int, _c_dbl, _c_int, _P, _P, _c_i64, _P]
    L.rt_build_batch.argtypes = [_P, _c_i64, ctypes.POINTER(RtHparams), _c_int, _c_int, _P, ctypes.POINTER(_P)]
    L.rt_batch_info.argtypes = [_P, ctypes.POINTER(RtBatchInfo), _P, _P]
    L.rt_batch_apply.argtypes = [_P, _P, _P, _P]
    L.rt_solve_batch.argtypes = [_P, ctypes.POINTER(RtSolveOpts), _P, _P, _P, ctypes.POINTER(RtSolveStats), _P]
    L.rt_batch_set_wait.argtypes = [_P, _c_i64, _c_int]
    L.rt_batch_free.argtypes = [_P]
    L.rt_batch_free.restype = None
    L.rt_batch_last_error.restype = ctypes.c_char_p
    L.rt_server_create.argtypes = [ctypes.POINTER(RtServerOpts), ctypes.POINTER(_P)]
    L.rt_submit.argtypes = [_P, ctypes.POINTER(RtProblem), ctypes.POINTER(_c_i64)]
    L.rt_poll.argtypes = [_P, _c_i64, _c_int, _P, _P, ctypes.POINTER(RtRequestInfo)]
    L.rt_server_info.argtypes = [_P, ctypes.POINTER(RtServerInfo)]
    L.rt_server_free.argtypes = [_P]
    L.rt_server_free.restype = None
    _lib = L
    return L


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != RT_OK:
        raise RtError(rc, lib().rt_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return _P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def hparams(mode=RT_MODE_HMATRIX, prec=None, far_prec=RT_PREC_F32, aca_eps=1e-4, leaf=64, eta=2.0, gauss_pts=16,
            rank_max=0, adm=RT_ADM_GAP, line_eval=RT_LINE_CLOSED, refine=0, tensor_cores=0,
            wave_bytes=0, kappa_bins=0) -> RtHparams:
    if prec is None:
        prec = RT_PREC_F32
    return RtHparams(mode, prec, far_prec, aca_eps, leaf, eta, gauss_pts, rank_max, adm, line_eval, refine,
                     tensor_cores, int(wave_bytes), int(kappa_bins))


class _ProblemArgs:
    """Holds the C structs and the numpy arrays they point into."""

    def __init__(self, prob):
        self.xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
        self.tet = np.ascontiguousarray(prob.tet, dtype=np.int32)
        self.tri = np.ascontiguousarray(prob.emit_tri, dtype=np.int32).reshape(-1, 3)
        fr = prob.freqs
        self.nu = np.ascontiguousarray(fr.nu, dtype=np.float64)
        self.w = np.ascontiguousarray(fr.w, dtype=np.float64)
        self.c = np.ascontiguousarray(fr.c, dtype=np.float64)
        self.a = np.ascontiguousarray(fr.albedo, dtype=np.float64)
        grp = getattr(fr, "group", None)
        self.group = None if grp is None else np.ascontiguousarray(grp, dtype=np.int32)
        walls = ([] if prob.wall is None else [prob.wall]) + list(getattr(prob, "more_walls", ()) or ())
        self.walls = None
        n_walls = len(walls)
        if n_walls:
            self.walls = (RtWall * n_walls)()
            for k, wl in enumerate(walls):
                for d in range(3):
                    self.walls[k].p[d] = float(wl.p[d])
                    self.walls[k].n[d] = float(wl.n[d])
                self.walls[k].R0 = float(wl.R0)
        self.s = RtProblem()
        self.s.mesh = RtMesh(self.xyz.shape[0], _ptr(self.xyz), self.tet.shape[0], _ptr(self.tet))
        kap = prob.kappa
        self.s.kappa = RtKappa(int(kap.kind), float(kap.k0), float(kap.amp))
        grid = getattr(kap, "grid", None)
        self.grid = None
        if grid is not None:
            self.grid = np.ascontiguousarray(grid, dtype=np.float32)   # [nz, ny, nx], x fastest
            nz, ny, nx = self.grid.shape
            self.s.kappa.grid = _ptr(self.grid)
            self.s.kappa.dims[0], self.s.kappa.dims[1], self.s.kappa.dims[2] = nx, ny, nz
            for d in range(6):
                self.s.kappa.bbox[d] = float(kap.bbox[d])
        obst = list(getattr(prob, "obstacles", ()) or ())
        self.obst = None
        if obst:
            self.obst = (RtBox * len(obst))()
            for o, b in enumerate(obst):
                for d in range(3):
                    self.obst[o].lo[d] = float(b.lo[d])
                    self.obst[o].hi[d] = float(b.hi[d])
            self.s.n_obstacles = len(obst)
            self.s.obstacles = ctypes.cast(self.obst, _P)
        self.s.n_walls = n_walls
        self.s.walls = ctypes.cast(self.walls, _P) if self.walls is not None else None
        self.s.n_emit = self.tri.shape[0]
        self.s.emit_tri = _ptr(self.tri)
        self.s.Q0 = float(prob.Q0)
        self.s.T_emit = float(prob.T_emit)
        self.s.grey = 1 if prob.grey else 0
        self.s.freqs = RtFreqs(self.nu.shape[0], _ptr(self.nu), _ptr(self.w), _ptr(self.c), _ptr(self.a),
                               _ptr(self.group) if self.group is not None else None)
        self.s.corner = 1 if getattr(prob, "corner", False) else 0


class Operator:
    """A built operator (owned by the library; released by :meth:`free`)."""

    def __init__(self, handle, N, F, vec64):
        self.h = handle
        self.N = N
        self.F = F
        self.vec64 = vec64

    def info(self) -> dict:
        i = RtInfo()
        _check(lib().rt_operator_info(self.h, ctypes.byref(i)))
        return i.as_dict()

    def apply(self, X, Y, stream=None):
        """rt_apply: Y = Gbar X, torch tensors [F, N] on the device."""
        _check(lib().rt_apply(self.h, _P(X.data_ptr()), _P(Y.data_ptr()), _stream_ptr(stream)))

    def apply_group(self, group, X, Y, nrhs=None, ldx=None, ldy=None, stream=None):
        """rt_apply_group: Y_j = G_group X_j for nrhs vectors (rows of X, Y with leading dimensions)."""
        nrhs = X.shape[0] if nrhs is None else nrhs
        ldx = X.stride(0) if ldx is None else ldx
        ldy = Y.stride(0) if ldy is None else ldy
        _check(lib().rt_apply_group(self.h, int(group), _P(X.data_ptr()), int(ldx), int(nrhs), _P(Y.data_ptr()),
                                    int(ldy), _stream_ptr(stream)))

    def apply_noalloc(self, X, Y, stream=None):
        """rt_apply_noalloc: Y = Gbar X using the library's static scratch array (no allocation)."""
        _check(lib().rt_apply_noalloc(self.h, _P(X.data_ptr()), _P(Y.data_ptr()), _stream_ptr(stream)))

    def source(self, out, stream=None):
        """rt_source: Sbar^E into out [F, N]."""
        _check(lib().rt_source(self.h, _P(out.data_ptr()), _stream_ptr(stream)))

    def eval_entries(self, group, rows, cols, out, stream=None):
        """rt_eval_entries: out[k] = G_group[rows[k], cols[k]] (device int32 rows/cols, float64 out)."""
        _check(lib().rt_eval_entries(self.h, int(group), int(rows.numel()), _P(rows.data_ptr()),
                                     _P(cols.data_ptr()), _P(out.data_ptr()), _stream_ptr(stream)))

    def solve_fixed_point(self, J, T, tol=1e-10, max_iter=500, check_every=1, T0=0.0, use_J0=False,
                          use_graph=True, stream=None, raise_on_noconv=True, refine_tol=0.0) -> dict:
        """rt_solve_fixed_point: J [F, N] and T [N] (float64) receive the final iterate."""
        o = RtSolveOpts(float(tol), int(max_iter), int(check_every), float(T0), 1 if use_J0 else 0,
                        1 if use_graph else 0, float(refine_tol))
        st = RtSolveStats()
        rc = lib().rt_solve_fixed_point(self.h, ctypes.byref(o), _P(J.data_ptr()), _P(T.data_ptr()),
                                        ctypes.byref(st), _stream_ptr(stream))
        d = st.as_dict()
        d["rc"] = rc
        if rc != RT_OK and (raise_on_noconv or rc != RT_ENOCONV):
            _check(rc)
        return d

    def free(self):
        if self.h:
            lib().rt_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rt_build_operator(prob, hp: RtHparams, stream=None) -> Operator:
    """Build the operator of one problem (any object with the attributes of
    ``workloads.Problem``: xyz, tet, emit_tri, kappa, wall, freqs, grey, Q0, T_emit)."""
    args = _ProblemArgs(prob)
    out = _P()
    _check(lib().rt_build_operator(ctypes.byref(args.s), ctypes.byref(hp), _stream_ptr(stream), ctypes.byref(out)))
    vec64 = hp.mode == RT_MODE_DENSE and hp.prec == RT_PREC_F64
    return Operator(out, args.xyz.shape[0], args.nu.shape[0], vec64)


class SourceOperator:
    """The surface-to-volume matrix Sbar^E_{i,l} of an operator (rt_build_source_operator)."""

    def __init__(self, handle, op):
        self.h = handle
        self.op = op   # the operator must outlive this one
        i = RtSourceInfo()
        _check(lib().rt_source_operator_info(self.h, ctypes.byref(i), None))
        self._info = i.as_dict()
        self.vertices = np.zeros(self._info["L"], dtype=np.int32)
        _check(lib().rt_source_operator_info(self.h, ctypes.byref(i), _ptr(self.vertices)))

    def info(self) -> dict:
        return dict(self._info)

    def apply(self, Q0, out, stream=None):
        """rt_apply_source: out [F, N] = B_nu(T_emit) Sbar^E_g Q0 for device Q0 [L] (float32)."""
        _check(lib().rt_apply_source(self.h, _P(Q0.data_ptr()), _P(out.data_ptr()), _stream_ptr(stream)))

    def free(self):
        if self.h:
            lib().rt_source_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rt_build_source_operator(op: "Operator", stream=None) -> SourceOperator:
    out = _P()
    _check(lib().rt_build_source_operator(op.h, _stream_ptr(stream), ctypes.byref(out)))
    return SourceOperator(out, op)


def rt_eval_sin2pi(x, lib_out, ref_out, stream=None):
    """rt_eval_sin2pi (diagnostic): the library's FP32 sin(2 pi x) and CUDA's sinpif(2x)."""
    _check(lib().rt_eval_sin2pi(_P(x.data_ptr()), _P(lib_out.data_ptr()), _P(ref_out.data_ptr()), x.numel(),
                                _stream_ptr(stream)))


def rt_plan(xyz, leaf=64, eta=2.0, adm=RT_ADM_GAP):
    """Host-only cluster/block tree: (perm [N], blocks [nb,5], counts (leaves, dense, admissible))."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    counts = np.zeros(3, dtype=np.int64)
    _check(lib().rt_plan(_ptr(xyz), n, int(leaf), float(eta), int(adm), None, None, 0, _ptr(counts)))
    perm = np.zeros(n, dtype=np.int32)
    nb = int(counts[1] + counts[2])
    blocks = np.zeros((max(nb, 1), 5), dtype=np.int32)
    _check(lib().rt_plan(_ptr(xyz), n, int(leaf), float(eta), int(adm), _ptr(perm), _ptr(blocks), nb,
                         _ptr(counts)))
    return perm, blocks[:nb], tuple(int(c) for c in counts)


def _check_batch(rc):
    if rc != RT_OK:
        raise RtError(rc, lib().rt_batch_last_error().decode(errors="replace"))


class Batch:
    """Independent instances applied and solved together (rt_build_batch)."""

    def __init__(self, handle, count):
        self.h = handle
        self.count = count
        i = RtBatchInfo()
        self.vec_off = np.zeros(count + 1, dtype=np.int64)
        self.vert_off = np.zeros(count + 1, dtype=np.int64)
        _check_batch(lib().rt_batch_info(self.h, ctypes.byref(i), _ptr(self.vec_off), _ptr(self.vert_off)))
        self._info = i.as_dict()

    def info(self) -> dict:
        return dict(self._info)

    def apply(self, X, Y, stream=None):
        """rt_batch_apply on concatenated [total_vec] float32 device tensors."""
        _check_batch(lib().rt_batch_apply(self.h, _P(X.data_ptr()), _P(Y.data_ptr()), _stream_ptr(stream)))

    def solve(self, J, T, tol=1e-6, max_iter=300, check_every=4, T0=0.0, use_graph=True, stream=None,
              raise_on_noconv=True):
        """rt_solve_batch: J [total_vec] float32, T [total_vert] float64 device tensors; returns (iters, stats)."""
        o = RtSolveOpts(float(tol), int(max_iter), int(check_every), float(T0), 0, 1 if use_graph else 0, 0.0)
        st = RtSolveStats()
        iters = np.zeros(self.count, dtype=np.int32)
        rc = lib().rt_solve_batch(self.h, ctypes.byref(o), _P(J.data_ptr()), _P(T.data_ptr()), _ptr(iters),
                                  ctypes.byref(st), _stream_ptr(stream))
        if rc != RT_OK and (raise_on_noconv or rc != RT_ENOCONV):
            _check_batch(rc)
        return iters, st.as_dict()

    def set_wait(self, wait_cycles: int = 0, unreachable: bool = False):
        """rt_batch_set_wait (diagnostic): budget of the phase-2 waits; unreachable makes them run out."""
        _check_batch(lib().rt_batch_set_wait(self.h, int(wait_cycles), 1 if unreachable else 0))

    def free(self):
        if self.h:
            lib().rt_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rt_build_batch(problems, hp: RtHparams, threads: int = 8, tune: bool = True, stream=None) -> Batch:
    """Build one operator per problem and the batch structures (rt_build_batch)."""
    args = [_ProblemArgs(p) for p in problems]
    arr = (RtProblem * len(args))(*[a.s for a in args])
    out = _P()
    _check_batch(lib().rt_build_batch(ctypes.cast(arr, _P), len(args), ctypes.byref(hp), int(threads),
                                      1 if tune else 0, _stream_ptr(stream), ctypes.byref(out)))
    return Batch(out, len(args))



class Server:
    """Continuous admission of solve requests under an HBM budget (rt_server_create).

    ``submit`` copies a problem and returns at once with an id; ``poll`` returns
    None while the request is queued or running, else (J [F, N] float32 numpy,
    T [N] float64 numpy, info dict)."""

    def __init__(self, hp: RtHparams, hbm_budget=120 * 10**9, slots=8, max_bypass=4, tol=1e-6, max_iter=300,
                 check_every=4, T0=0.0, use_graph=True, refine_tol=0.0):
        o = RtServerOpts(int(hbm_budget), int(slots), int(max_bypass), hp,
                         RtSolveOpts(float(tol), int(max_iter), int(check_every), float(T0), 0,
                                     1 if use_graph else 0, float(refine_tol)))
        self.h = _P()
        _check(lib().rt_server_create(ctypes.byref(o), ctypes.byref(self.h)))
        self._dims = {}

    def submit(self, prob) -> int:
        a = _ProblemArgs(prob)
        rid = _c_i64(0)
        _check(lib().rt_submit(self.h, ctypes.byref(a.s), ctypes.byref(rid)))
        self._dims[rid.value] = (prob.freqs.F, prob.N)
        return rid.value

    def poll(self, rid: int, wait_ms: int = 0, raise_on_error=True):
        F, N = self._dims[rid]
        J = np.empty((F, N), dtype=np.float32)
        T = np.empty(N, dtype=np.float64)
        info = RtRequestInfo()
        rc = lib().rt_poll(self.h, int(rid), int(wait_ms), _ptr(J), _ptr(T), ctypes.byref(info))
        if rc == RT_EAGAIN:
            return None
        del self._dims[rid]
        d = info.as_dict()
        if rc != RT_OK and raise_on_error:
            _check(rc)
        return J, T, d

    def info(self) -> dict:
        i = RtServerInfo()
        _check(lib().rt_server_info(self.h, ctypes.byref(i)))
        return i.as_dict()

    def free(self):
        if self.h:
            lib().rt_server_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
