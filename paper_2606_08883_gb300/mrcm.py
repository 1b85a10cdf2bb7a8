"""ctypes binding of libmrcm (include/mrcm.h): the same entry-point names, argument marshalling only.

Every numerical step runs inside the library's CUDA kernels; PyTorch supplies device memory (the
workspace and the caller's arrays) and streams.  Importing this module loads the in-tree
``_lib/libmrcm.so`` and raises ImportError if it has not been built (there is no fallback).

``Solver`` is a convenience wrapper that owns the workspace and the device copies of a
``workloads.Problem``.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libmrcm.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libmrcm is not built ({_LIB_PATH} missing); run paper_2606_08883_gb300.build.build()")
_lib = C.CDLL(_LIB_PATH)

MRCM_OK, MRCM_ERR_INVALID_ARG, MRCM_ERR_OOM, MRCM_ERR_SINGULAR, MRCM_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
MRCM_SMOOTH_ADDITIVE, MRCM_SMOOTH_MULTIPLICATIVE = 0, 1
MRCM_ERR_TIMEOUT, MRCM_ERR_CUDA, MRCM_ERR_BUSY, MRCM_ERR_UNSUPPORTED, MRCM_ERR_CANCELLED = 5, 6, 7, 8, 9
MRCM_BC_DIRICHLET, MRCM_BC_NEUMANN = 0, 1
MRCM_PREC_FP64, MRCM_PREC_FP32 = 0, 1
MRCM_DBG_TRANS, MRCM_DBG_PHI, MRCM_DBG_PSI, MRCM_DBG_MOMENTS, MRCM_DBG_G, MRCM_DBG_COARSE, MRCM_DBG_ZMRCM = range(7)
COARSE_METHODS = ("inverse", "band", "band_pivoted", "multifrontal")   # mrcm_coarse_method codes


class mrcm_problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("h", C.c_double * 3), ("K", C.c_void_p),
                ("bc_kind", C.c_int32 * 6), ("bc_val", C.c_void_p * 6), ("f", C.c_void_p),
                ("K_y", C.c_void_p), ("K_z", C.c_void_p)]


class mrcm_params(C.Structure):
    _fields_ = [("sub", C.c_int32 * 3), ("oversample", C.c_int32), ("smooth_steps", C.c_int32),
                ("alpha", C.c_double), ("tol", C.c_double), ("tol_relative", C.c_int32),
                ("restart", C.c_int32), ("max_iter", C.c_int32), ("local_prec", C.c_int32),
                ("smooth_kind", C.c_int32), ("iface_degree", C.c_int32), ("coarse_pivoting", C.c_int32),
                ("refine_setup", C.c_int32),
                ("coarse_solver", C.c_int32)]


class mrcm_result(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32),
                ("history_len", C.c_int32), ("abs_res", C.c_double), ("rel_res", C.c_double),
                ("bnorm", C.c_double), ("history", C.POINTER(C.c_double)), ("history_cap", C.c_int32),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double)]


_P, _Q, _R = C.POINTER(mrcm_problem), C.POINTER(mrcm_params), C.POINTER(mrcm_result)
_H = C.c_void_p
_SIGS = {
    "mrcm_footprint": ([_P, _Q, C.POINTER(C.c_size_t)], C.c_int),
    "mrcm_setup": ([_P, _Q, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(_H)], C.c_int),
    "mrcm_update_problem": ([_H, _P, C.c_void_p], C.c_int),
    "mrcm_factor_local": ([_H, C.c_void_p], C.c_int),
    "mrcm_apply_precond": ([_H, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mrcm_apply_operator": ([_H, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mrcm_rhs": ([_H, C.c_void_p, C.c_void_p], C.c_int),
    "mrcm_gmres_solve": ([_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _R, C.c_void_p], C.c_int),
    "mrcm_solve_host": ([_H, C.c_void_p, C.c_void_p, _R, C.c_void_p], C.c_int),
    "mrcm_destroy": ([_H], None),
    "mrcm_status_string": ([C.c_int], C.c_char_p),
    "mrcm_last_error": ([_H], C.c_char_p),
    "mrcm_plan_export": ([_P, _Q, C.POINTER(C.c_int32), C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "mrcm_plan_mf_export": ([_P, _Q, C.POINTER(C.c_int32), C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "mrcm_debug_get": ([_H, C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t), C.c_void_p], C.c_int),
    "mrcm_profile_enable": ([_H, C.c_int32], C.c_int),
    "mrcm_profile_select": ([_H, C.c_uint32, C.c_int32], C.c_int),
    "mrcm_profile_read": ([_H, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32, C.c_int32, C.c_void_p], C.c_int),
    "mrcm_launch_count": ([], C.c_int64),
    "mrcm_measure_fp64_peak": ([C.POINTER(C.c_double), C.c_void_p], C.c_int32),
    "mrcm_coarse_method": ([_H, C.POINTER(C.c_int32)], C.c_int32),
    "mrcm_residual_norm_noalloc": ([_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "mrcm_server_create": ([C.c_void_p, C.c_size_t, C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "mrcm_submit": ([C.c_void_p, _P, _Q, C.POINTER(C.c_uint64)], C.c_int),
    "mrcm_poll": ([C.c_void_p, C.c_uint64, C.c_void_p, _R, C.POINTER(C.c_int32)], C.c_int),
    "mrcm_cancel": ([C.c_void_p, C.c_uint64], C.c_int),
    "mrcm_server_stats": ([C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_size_t,
                           C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
    "mrcm_server_destroy": ([C.c_void_p], None),
    "mrcm_autotune": ([C.c_int32], None),
    "mrcm_autotune_table": ([C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
}
PHASES = ("assemble", "factor_ohat_robin", "informed", "factor_omega", "basis", "coarse_factor",
          "factor_ohat_dirichlet", "particular", "coarse_solve", "reconstruct", "residual", "schwarz", "krylov", "stage")
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res
    globals()[_name] = _fn

EXPORTED = tuple(_SIGS)


def autotune(mode):
    """0 off, 1 on (the default), 2 forget the tuned shapes and turn on."""
    mrcm_autotune(int(mode))


def autotune_table():
    """The tuned launch shapes: list of dicts (kind, key, choice, ncand, best_us)."""
    n = C.c_size_t()
    _check(mrcm_autotune_table(None, 0, C.byref(n)))
    buf = (C.c_double * max(n.value, 1))()
    _check(mrcm_autotune_table(buf, n.value, C.byref(n)))
    out = []
    for i in range(0, n.value, 10):
        e = buf[i:i + 10]
        out.append({"kind": int(e[0]), "key": tuple(int(v) for v in e[1:7]), "choice": int(e[7]),
                    "ncand": int(e[8]), "best_us": float(e[9])})
    return out


def measure_fp64_peak(stream=None):
    """Measured FP64 FMA throughput of the current device, TFLOP/s (mrcm_measure_fp64_peak)."""
    v = C.c_double(0.0)
    _check(mrcm_measure_fp64_peak(C.byref(v), _stream_ptr(stream)))
    return v.value


class MRCMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{mrcm_status_string(status).decode()}: {msg}")
        self.status = status


def _check(rc, handle=None):
    if rc != MRCM_OK:
        raise MRCMError(rc, (mrcm_last_error(handle) or b"").decode())
    return rc


def make_params(params):
    q = mrcm_params()
    q.sub[:] = [int(v) for v in params.sub]
    q.oversample = int(params.oversample)
    q.smooth_steps = int(params.smooth_steps)
    q.alpha = float(params.alpha)
    q.tol = float(params.tol)
    q.tol_relative = int(params.tol_relative)
    q.restart = int(params.restart)
    q.max_iter = int(params.max_iter)
    q.local_prec = int(params.local_prec)
    q.smooth_kind = int(getattr(params, "smooth_kind", 0))
    q.iface_degree = int(getattr(params, "iface_degree", 0))
    q.coarse_pivoting = int(getattr(params, "coarse_pivoting", 0))
    q.refine_setup = int(getattr(params, "refine_setup", 0))
    q.coarse_solver = int(getattr(params, "coarse_solver", 0))
    return q


def make_problem(problem, K_ptr=0, bc_ptrs=None, f_ptr=0, Ky_ptr=0):
    p = mrcm_problem()
    p.dim = int(problem.dim)
    p.n[:] = [int(v) for v in problem.n]
    p.h[:] = [float(v) for v in problem.h]
    p.K = K_ptr or None
    p.bc_kind[:] = [int(v) for v in problem.bc_kind]
    ptrs = bc_ptrs or [0] * 6
    for s in range(6):
        p.bc_val[s] = ptrs[s] or None
    p.f = f_ptr or None
    p.K_y = Ky_ptr or None
    p.K_z = None
    return p


def plan_export(problem, params):
    """Integer partition tables (host only, no GPU needed)."""
    p, q = make_problem(problem), make_params(params)
    n = C.c_size_t(0)
    _check(mrcm_plan_export(C.byref(p), C.byref(q), None, 0, C.byref(n)))
    buf = np.zeros(n.value, dtype=np.int32)
    _check(mrcm_plan_export(C.byref(p), C.byref(q), buf.ctypes.data_as(C.POINTER(C.c_int32)), n.value, C.byref(n)))
    return buf


def plan_mf_export(problem, params):
    """The multifrontal plan of the coupling factorisation (host only, no GPU needed): a dict with
    'used', 'NC', 'kl', 'ku', 'fronts' (list of dicts np, nu, level, children, parent, unknowns,
    entries as (row, column) pairs of G)."""
    p, q = make_problem(problem), make_params(params)
    n = C.c_size_t(0)
    _check(mrcm_plan_mf_export(C.byref(p), C.byref(q), None, 0, C.byref(n)))
    buf = np.zeros(n.value, dtype=np.int32)
    _check(mrcm_plan_mf_export(C.byref(p), C.byref(q), buf.ctypes.data_as(C.POINTER(C.c_int32)), n.value,
                               C.byref(n)))
    used, nf, levels, NC, kl, ku = (int(v) for v in buf[:6])
    o = 6
    fronts = []
    for f in range(nf):
        np_, nu, lev, nch, c0, c1, par = (int(v) for v in buf[o:o + 7])
        fronts.append(dict(np=np_, nu=nu, level=lev, children=[c for c in (c0, c1)[:nch]], parent=par))
        o += 7
    for fr in fronts:
        k = fr["np"] + fr["nu"]
        fr["unknowns"] = buf[o:o + k].astype(np.int64)
        o += k
    for fr in fronts:
        na = int(buf[o])
        fr["entries"] = buf[o + 1:o + 1 + 2 * na].reshape(na, 2).astype(np.int64)
        o += 1 + 2 * na
    return dict(used=bool(used), NC=NC, kl=kl, ku=ku, levels=levels, fronts=fronts)


def footprint(problem, params):
    p, q = make_problem(problem), make_params(params)
    n = C.c_size_t(0)
    _check(mrcm_footprint(C.byref(p), C.byref(q), C.byref(n)))
    return n.value


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Solver:
    """Owns the workspace and device copies of a ``workloads.Problem`` (float64 tensors)."""

    def __init__(self, problem, params, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.problem, self.params = problem, params
        self.device = torch.device(device)
        self.stream = stream
        self.n = int(np.prod(problem.n))
        self._upload(problem)
        self.q = make_params(params)
        self.bytes = footprint(problem, params)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.handle = _H()
        _check(mrcm_setup(C.byref(self.p), C.byref(self.q), C.c_void_p(self._ws_ptr), self.bytes,
                          _stream_ptr(stream), C.byref(self.handle)))

    def _upload(self, problem):
        t = self.torch
        K = np.asarray(problem.K, dtype=np.float64)  # scalar field, or diagonal tensor components stacked first
        self.K = t.as_tensor(np.ascontiguousarray(K[0] if K.ndim == 4 else K).ravel(), device=self.device)
        self.Ky = t.as_tensor(np.ascontiguousarray(K[1]).ravel(), device=self.device) if K.ndim == 4 else None
        self.bc = [None if v is None else t.as_tensor(np.ascontiguousarray(v, dtype=np.float64).ravel(),
                                                      device=self.device) for v in problem.bc_val]
        self.f = None if problem.f is None else t.as_tensor(np.ascontiguousarray(problem.f, dtype=np.float64).ravel(),
                                                             device=self.device)
        self.p = make_problem(problem, self.K.data_ptr(), [0 if v is None else v.data_ptr() for v in self.bc],
                              0 if self.f is None else self.f.data_ptr(),
                              0 if self.Ky is None else self.Ky.data_ptr())

    def update(self, problem):
        self._upload(problem)
        _check(mrcm_update_problem(self.handle, C.byref(self.p), _stream_ptr(self.stream)), self.handle)

    def factor(self):
        _check(mrcm_factor_local(self.handle, _stream_ptr(self.stream)), self.handle)

    def empty(self):
        return self.torch.empty(self.n, dtype=self.torch.float64, device=self.device)

    def apply_precond(self, r, z=None):
        z = self.empty() if z is None else z
        _check(mrcm_apply_precond(self.handle, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()),
                                  _stream_ptr(self.stream)), self.handle)
        return z

    def apply_operator(self, v, w=None):
        w = self.empty() if w is None else w
        _check(mrcm_apply_operator(self.handle, C.c_void_p(v.data_ptr()), C.c_void_p(w.data_ptr()),
                                   _stream_ptr(self.stream)), self.handle)
        return w

    def rhs(self):
        b = self.empty()
        _check(mrcm_rhs(self.handle, C.c_void_p(b.data_ptr()), _stream_ptr(self.stream)), self.handle)
        return b

    def solve(self, b=None, p=None, fluxes=False, history_cap=4096, allow_not_converged=False):
        t = self.torch
        p = t.zeros(self.n, dtype=t.float64, device=self.device) if p is None else p
        nx, ny = self.problem.n[0], self.problem.n[1]
        ux = t.empty((nx + 1) * ny, dtype=t.float64, device=self.device) if fluxes else None
        uy = t.empty(nx * (ny + 1), dtype=t.float64, device=self.device) if fluxes else None
        hist = (C.c_double * history_cap)()
        res = mrcm_result()
        res.history = C.cast(hist, C.POINTER(C.c_double))
        res.history_cap = history_cap
        rc = mrcm_gmres_solve(self.handle, C.c_void_p(b.data_ptr()) if b is not None else None,
                              C.c_void_p(p.data_ptr()), C.c_void_p(ux.data_ptr()) if fluxes else None,
                              C.c_void_p(uy.data_ptr()) if fluxes else None, None, C.byref(res),
                              _stream_ptr(self.stream))
        if rc != MRCM_OK and not (allow_not_converged and rc == MRCM_ERR_NOT_CONVERGED):
            _check(rc, self.handle)
        info = {"iterations": res.iterations, "restarts": res.restarts, "status": res.status,
                "abs_res": res.abs_res, "rel_res": res.rel_res, "bnorm": res.bnorm,
                "history": [hist[i] for i in range(res.history_len)]}
        if fluxes:
            info["u"] = (ux, uy)
        return p, info

    def solve_host(self, K_host, p_host):
        """End-to-end: host K in, host p out (numpy float64 arrays, ideally pinned)."""
        res = mrcm_result()
        rc = mrcm_solve_host(self.handle, C.c_void_p(K_host.data_ptr()) if K_host is not None else None,
                             C.c_void_p(p_host.data_ptr()), C.byref(res), _stream_ptr(self.stream))
        if rc not in (MRCM_OK, MRCM_ERR_NOT_CONVERGED):
            _check(rc, self.handle)
        return {"iterations": res.iterations, "abs_res": res.abs_res, "rel_res": res.rel_res, "status": res.status}

    def coarse_method(self):
        """How the last factor() factored G: one of COARSE_METHODS (mrcm_coarse_method)."""
        v = C.c_int32(-1)
        _check(mrcm_coarse_method(self.handle, C.byref(v)), self.handle)
        return COARSE_METHODS[v.value]

    def debug(self, what, enable_only=False):
        n = C.c_size_t(0)
        if enable_only:
            _check(mrcm_debug_get(self.handle, what, None, 0, C.byref(n), _stream_ptr(self.stream)), self.handle)
            return None
        _check(mrcm_debug_get(self.handle, what, None, 0, C.byref(n), _stream_ptr(self.stream)), self.handle)
        out = np.zeros(n.value, dtype=np.float64)
        _check(mrcm_debug_get(self.handle, what, C.c_void_p(out.ctypes.data), n.value, C.byref(n),
                              _stream_ptr(self.stream)), self.handle)
        return out

    def profile(self, enable=True, phases=None, every=1):
        """Per-phase event timing on or off; ``phases`` (names from PHASES) restricts the recording
        to those phases (None: all), ``every`` to every every-th occurrence of each."""
        mask = 0xFFFFFFFF if phases is None else sum(1 << PHASES.index(p) for p in phases)
        _check(mrcm_profile_select(self.handle, mask, int(every)), self.handle)
        _check(mrcm_profile_enable(self.handle, 1 if enable else 0), self.handle)

    def profile_read(self, reset=True):
        """{phase: (milliseconds, launches)} accumulated since the last reset."""
        ms = (C.c_double * len(PHASES))()
        nl = (C.c_int64 * len(PHASES))()
        _check(mrcm_profile_read(self.handle, ms, nl, len(PHASES), 1 if reset else 0, _stream_ptr(self.stream)),
               self.handle)
        return {name: (ms[i], nl[i]) for i, name in enumerate(PHASES)}

    def close(self):
        if getattr(self, "handle", None):
            mrcm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server over a caller-owned device arena (a torch tensor)."""

    def __init__(self, arena_bytes, max_inflight=4, device="cuda"):
        import torch
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8, device=device)
        base = (self.arena.data_ptr() + 255) // 256 * 256
        self.handle = C.c_void_p()
        _check(mrcm_server_create(C.c_void_p(base), arena_bytes, max_inflight, C.byref(self.handle)))
        self._keep = {}

    def submit(self, problem, params):
        """Queue a solve of a ``workloads.Problem`` (host numpy data); returns the ticket."""
        Kall = np.asarray(problem.K, dtype=np.float64)
        K = np.ascontiguousarray(Kall[0] if Kall.ndim == 4 else Kall).ravel()
        Ky = np.ascontiguousarray(Kall[1]).ravel() if Kall.ndim == 4 else None
        bcs = [None if v is None else np.ascontiguousarray(v, dtype=np.float64).ravel() for v in problem.bc_val]
        f = None if problem.f is None else np.ascontiguousarray(problem.f, dtype=np.float64).ravel()
        p = make_problem(problem, K.ctypes.data, [0 if v is None else v.ctypes.data for v in bcs],
                         0 if f is None else f.ctypes.data, 0 if Ky is None else Ky.ctypes.data)
        q = make_params(params)
        t = C.c_uint64()
        _check(mrcm_submit(self.handle, C.byref(p), C.byref(q), C.byref(t)))
        self._keep[t.value] = int(np.prod(problem.n))
        return t.value

    def poll(self, ticket, history_cap=0):
        """None while running; else (status, p (numpy), info)."""
        n = self._keep[ticket]
        p = np.empty(n)
        hist = (C.c_double * max(history_cap, 1))()
        res = mrcm_result()
        res.history = C.cast(hist, C.POINTER(C.c_double)) if history_cap else None
        res.history_cap = history_cap
        done = C.c_int32(0)
        rc = mrcm_poll(self.handle, ticket, C.c_void_p(p.ctypes.data), C.byref(res), C.byref(done))
        if not done.value:
            if rc != MRCM_OK:
                _check(rc)
            return None
        del self._keep[ticket]
        info = {"iterations": res.iterations, "restarts": res.restarts, "abs_res": res.abs_res,
                "rel_res": res.rel_res, "latency_ms": res.latency_ms, "queue_ms": res.queue_ms,
                "history": [hist[i] for i in range(res.history_len)]}
        if rc != MRCM_OK:
            info["error"] = (mrcm_last_error(None) or b"").decode()
        return rc, p, info

    def cancel(self, ticket):
        _check(mrcm_cancel(self.handle, ticket))

    def stats(self):
        counts = (C.c_int64 * 5)()
        n = C.c_size_t(0)
        peak = C.c_size_t(0)
        _check(mrcm_server_stats(self.handle, counts, None, 0, C.byref(n), C.byref(peak)))
        lat = (C.c_double * max(n.value, 1))()
        _check(mrcm_server_stats(self.handle, counts, lat, n.value, C.byref(n), C.byref(peak)))
        keys = ("submitted", "queued", "running", "completed", "failed")
        out = {k: counts[i] for i, k in enumerate(keys)}
        out["latency_ms"] = [lat[i] for i in range(n.value)]
        out["arena_peak"] = peak.value
        return out

    def close(self):
        if getattr(self, "handle", None):
            mrcm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
