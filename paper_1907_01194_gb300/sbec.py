"""Python binding of libsbec (argument marshalling only).

Every computation runs in the compiled CUDA library; this module converts
arguments (torch tensors on the GPU, or numpy arrays on the host) to plain
pointers and sizes and forwards the call through the C ABI declared in
include/sbec.h.  Importing it loads the library and raises ImportError if it
has not been built; there is no fallback implementation.

Arrays use the library's layout: complex tensors of shape (C, n_z, n_y, n_x)
(1D: (C, n_x), 2D: (C, n_y, n_x)), components l = F..-F, holding the paper's
scaled variable X = sqrt(dV) phi; complex128 for precision "fp64", complex64
for "mixed".
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SBEC_LIB", os.path.join(_HERE, "libsbec.so"))

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsbec is not built ({LIB_PATH} missing): run "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_DOMAIN, ERR_NONFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_NOCONV = range(7)
FP64, MIXED = 0, 1
S_ENERGY, S_RGRAD_NORM2, S_ALPHA_G, S_BETA_G, S_MASS, S_MAG, S_STATUS = range(7)


class Problem(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int), ("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("beta", ctypes.c_double * 4), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("M", ctypes.c_double), ("precision", ctypes.c_int)]


_vp, _dp, _int, _dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
_lib.sbec_create.argtypes = [ctypes.POINTER(Problem), _vp, _vp, ctypes.POINTER(_vp)]
_lib.sbec_destroy.argtypes = [_vp]
_lib.sbec_energy.argtypes = [_vp, _vp, _dp]
_lib.sbec_grad.argtypes = [_vp, _vp, _vp, _vp, _dp, _dp]
_lib.sbec_hessvec.argtypes = [_vp, _vp, _vp, _dbl, _int, _vp]
_lib.sbec_retract.argtypes = [_vp, _vp, _vp, _dbl, _int, _vp]
_lib.sbec_sync.argtypes = [_vp]
_lib.sbec_scalars.argtypes = [_vp]
_lib.sbec_scalars.restype = _vp
_lib.sbec_create_batch.argtypes = [ctypes.POINTER(Problem), _int, _vp, _vp, ctypes.POINTER(_vp)]
_lib.sbec_create_batch.restype = _int
_lib.sbec_batch_size.argtypes = [_vp]
_lib.sbec_batch_size.restype = _int
_lib.sbec_launch_count.argtypes = [_vp]
_lib.sbec_launch_count.restype = ctypes.c_longlong
_lib.sbec_profile.argtypes = [_vp, _int]
_lib.sbec_profile_read.argtypes = [_vp, _int, ctypes.c_char_p, _dp, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(_int)]
_lib.sbec_status_string.argtypes = [_int]
_lib.sbec_status_string.restype = ctypes.c_char_p
for _f in ("sbec_create", "sbec_destroy", "sbec_energy", "sbec_grad", "sbec_hessvec",
           "sbec_retract", "sbec_sync", "sbec_profile", "sbec_profile_read"):
    getattr(_lib, _f).restype = _int

EXPORTED = ("sbec_create", "sbec_destroy", "sbec_energy", "sbec_grad", "sbec_hessvec",
            "sbec_retract", "sbec_sync", "sbec_scalars", "sbec_status_string",
            "sbec_launch_count", "sbec_profile", "sbec_profile_read", "sbec_probe_fma_peak")


class SbecError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.sbec_status_string(status).decode()} (status {status})")


def _check(status, where):
    if status != OK:
        raise SbecError(status, where)


def _ptr(a):
    """Plain pointer of a contiguous torch tensor (device or host) or numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


class Handle:
    """One problem on the current CUDA device (sbec_create / sbec_destroy)."""

    def __init__(self, F, n, lo, hi, beta, M, p=0.0, q=0.0, V=None, precision="fp64",
                 stream=None):
        n = tuple(int(v) for v in n)
        dim = len(n)
        pr = Problem()
        pr.F, pr.dim = int(F), dim
        for i in range(3):
            pr.n[i] = n[i] if i < dim else 1
            pr.lo[i] = float(lo[i]) if i < dim else 0.0
            pr.hi[i] = float(hi[i]) if i < dim else 1.0
        b = tuple(beta) + (0.0,) * (4 - len(beta))
        for i in range(4):
            pr.beta[i] = float(b[i])
        pr.p, pr.q, pr.M = float(p), float(q), float(M)
        pr.precision = FP64 if precision == "fp64" else MIXED
        self.problem = pr
        self.F, self.C, self.n, self.dim = int(F), 2 * int(F) + 1, n, dim
        self.precision = precision
        self.shape = (self.C,) + tuple(reversed(n))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        if V is not None:
            if isinstance(V, np.ndarray):
                V = np.ascontiguousarray(V, dtype=np.float64)
            self._V_keep = V
        out = _vp()
        _check(_lib.sbec_create(ctypes.byref(pr), _ptr(V) if V is not None else None, stream,
                                ctypes.byref(out)), "sbec_create")
        self._h = out
        self.B = 1

    @classmethod
    def batch(cls, workloads, precision="fp64", V="auto", stream=None):
        """One batch handle (sbec_create_batch) for workloads that share spin, grid, box and
        Zeeman terms; arrays are then (B, C, ...) and scalar outputs have B entries."""
        from . import workloads as W
        ws = list(workloads)
        B = len(ws)
        probs = (Problem * B)()
        for i, w in enumerate(ws):
            n = tuple(int(v) for v in w.n)
            dim = len(n)
            pr = probs[i]
            pr.F, pr.dim = int(w.F), dim
            for a in range(3):
                pr.n[a] = n[a] if a < dim else 1
                pr.lo[a] = float(w.lo[a]) if a < dim else 0.0
                pr.hi[a] = float(w.hi[a]) if a < dim else 1.0
            b = tuple(w.beta) + (0.0,) * (4 - len(w.beta))
            for a in range(4):
                pr.beta[a] = float(b[a])
            pr.p, pr.q, pr.M = float(w.p), float(w.q), float(w.M)
            pr.precision = FP64 if precision == "fp64" else MIXED
        if isinstance(V, str) and V == "auto":
            V = np.ascontiguousarray(np.stack([W.potential(w) for w in ws]), dtype=np.float64)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self = cls.__new__(cls)
        self.problem = probs[0]
        self.F, self.C, self.n, self.dim = int(ws[0].F), ws[0].C, tuple(ws[0].n), len(ws[0].n)
        self.precision = precision
        self.shape = (B, self.C) + tuple(reversed(self.n))
        self.stream = stream
        self._V_keep = V
        out = _vp()
        _check(_lib.sbec_create_batch(probs, B, _ptr(V) if V is not None else None, stream, ctypes.byref(out)),
               "sbec_create_batch")
        self._h = out
        self.B = B
        return self

    @classmethod
    def from_workload(cls, w, precision="fp64", V="auto", stream=None):
        from . import workloads as W
        if isinstance(V, str) and V == "auto":
            V = W.potential(w)
        return cls(w.F, w.n, w.lo, w.hi, w.beta, w.M, p=w.p, q=w.q, V=V,
                   precision=precision, stream=stream)

    def close(self):
        if getattr(self, "_h", None):
            _lib.sbec_destroy(self._h)
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

    # -- calls -------------------------------------------------------------
    def _out(self, arr):
        return arr[0] if self.B == 1 else np.array(arr[:])

    def energy(self, X, sync=True):
        """E_h(X); an array of B values for a batch handle."""
        E = (ctypes.c_double * self.B)()
        _check(_lib.sbec_energy(self._h, _ptr(X), E if sync else None), "sbec_energy")
        return self._out(E) if sync else None

    def grad(self, X, G_euc=None, G_riem=None, sync=True):
        """Returns (E, ||grad E||_2) when sync (arrays of B values for a batch handle),
        else None (values stay on the device)."""
        E, rn = (ctypes.c_double * self.B)(), (ctypes.c_double * self.B)()
        _check(_lib.sbec_grad(self._h, _ptr(X), _ptr(G_euc), _ptr(G_riem),
                              E if sync else None, rn if sync else None), "sbec_grad")
        return (self._out(E), self._out(rn)) if sync else None

    def hessvec(self, X, Z, HZ, sigma=0.0, riemannian=False):
        _check(_lib.sbec_hessvec(self._h, _ptr(X), _ptr(Z), float(sigma), int(bool(riemannian)),
                                 _ptr(HZ)), "sbec_hessvec")

    def retract(self, U, Xi, t, kind, out):
        _check(_lib.sbec_retract(self._h, _ptr(U), _ptr(Xi), float(t), int(kind), _ptr(out)),
               "sbec_retract")

    def sync(self):
        _check(_lib.sbec_sync(self._h), "sbec_sync")

    def sync_status(self):
        return _lib.sbec_sync(self._h)

    def scalars_ptr(self):
        return _lib.sbec_scalars(self._h)

    def launch_count(self):
        return int(_lib.sbec_launch_count(self._h))

    def profile(self, enable=True):
        _check(_lib.sbec_profile(self._h, int(bool(enable))), "sbec_profile")

    def profile_read(self):
        """{kernel name: (total ms, launches)} of the launches recorded since profile(True)."""
        mx = 64
        names = ctypes.create_string_buffer(32 * mx)
        ms = (ctypes.c_double * mx)()
        cnt = (ctypes.c_longlong * mx)()
        rows = _int()
        _check(_lib.sbec_profile_read(self._h, mx, names, ms, cnt, ctypes.byref(rows)),
               "sbec_profile_read")
        out = {}
        for r in range(rows.value):
            nm = names.raw[32 * r: 32 * r + 32].split(b"\0", 1)[0].decode()
            out[nm] = (ms[r], int(cnt[r]))
        return out


class Tune(ctypes.Structure):
    _fields_ = [("x_rows", ctypes.c_int), ("s_pencils", ctypes.c_int * 3), ("s_split", ctypes.c_int * 3),
                ("elem_per_sm", ctypes.c_int), ("ms", ctypes.c_double)]


_lib.sbec_autotune.argtypes = [_vp, _vp, _int, ctypes.POINTER(Tune)]
_lib.sbec_autotune.restype = _int
_lib.sbec_set_tune.argtypes = [_vp, ctypes.POINTER(Tune)]
_lib.sbec_set_tune.restype = _int
_lib.sbec_get_tune.argtypes = [_vp, ctypes.POINTER(Tune)]
_lib.sbec_get_tune.restype = _int


def _tune_dict(t):
    return {"x_rows": t.x_rows, "s_pencils": list(t.s_pencils), "s_split": list(t.s_split),
            "elem_per_sm": t.elem_per_sm, "ms": t.ms}


def _autotune(self, X, reps=0):
    """sbec_autotune at state X (device array): picks the launch shapes by timing,
    leaves the handle on them and returns them as a dict (with the measured ms)."""
    t = Tune()
    _check(_lib.sbec_autotune(self._h, _ptr(X), int(reps), ctypes.byref(t)), "sbec_autotune")
    return _tune_dict(t)


def _get_tune(self):
    """Launch shapes in use (sbec_get_tune)."""
    t = Tune()
    _check(_lib.sbec_get_tune(self._h, ctypes.byref(t)), "sbec_get_tune")
    return _tune_dict(t)


def _set_tune(self, d):
    """Set launch shapes from a dict like autotune()'s (missing keys: built-in choice)."""
    t = Tune()
    t.x_rows = int(d.get("x_rows", 0))
    for a, v in enumerate(d.get("s_pencils", [0, 0, 0])):
        t.s_pencils[a] = int(v)
    for a, v in enumerate(d.get("s_split", [0, 0, 0])):
        t.s_split[a] = int(v)
    t.elem_per_sm = int(d.get("elem_per_sm", 0))
    _check(_lib.sbec_set_tune(self._h, ctypes.byref(t)), "sbec_set_tune")


Handle.autotune = _autotune
Handle.get_tune = _get_tune
Handle.set_tune = _set_tune


def library_symbols():
    """Names of the exported entry points that resolve in the loaded library."""
    return [name for name in EXPORTED if hasattr(_lib, name)]


_lib.sbec_probe_fma_peak.argtypes = [_int, _int, _dp]
_lib.sbec_probe_fma_peak.restype = _int


def probe_fma_peak(precision="fp64", iters=None):
    """Measured FMA rate of the current device in GFLOP/s (sbec_probe_fma_peak):
    the FP64 rate bounds the FP64 form of the hot path."""
    fp64 = precision == "fp64"
    if iters is None:
        iters = 20000 if fp64 else 400000
    g = ctypes.c_double()
    _check(_lib.sbec_probe_fma_peak(FP64 if fp64 else MIXED, int(iters), ctypes.byref(g)), "sbec_probe_fma_peak")
    return g.value


_lib.sbec_energy_noalloc.argtypes = [ctypes.POINTER(Problem), _vp, _vp, _dp, _vp]
_lib.sbec_energy_noalloc.restype = _int


def _noalloc_problem(F, n, lo, hi, beta, M, p, q):
    n = tuple(int(v) for v in n)
    dim = len(n)
    pr = Problem()
    pr.F, pr.dim = int(F), dim
    for i in range(3):
        pr.n[i] = n[i] if i < dim else 1
        pr.lo[i] = float(lo[i]) if i < dim else 0.0
        pr.hi[i] = float(hi[i]) if i < dim else 1.0
    b = tuple(beta) + (0.0,) * (4 - len(beta))
    for i in range(4):
        pr.beta[i] = float(b[i])
    pr.p, pr.q, pr.M, pr.precision = float(p), float(q), float(M), FP64
    return pr


def energy_noalloc(F, n, lo, hi, beta, M, X, p=0.0, q=0.0, V=None, stream=None):
    """E_h(X) through sbec_energy_noalloc: no handle and no device allocation, for
    callers that cannot allocate device memory where they need the energy.  X and
    V (None: harmonic trap) must be contiguous device tensors (complex128 state,
    float64 potential); FP64 only."""
    import torch
    C, G = 2 * int(F) + 1, int(np.prod([int(v) for v in n]))
    # the kernels read X and V in place through raw pointers: check what they will read
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.complex128
            and X.is_contiguous() and X.numel() == C * G):
        raise ValueError(f"X must be a contiguous complex128 CUDA tensor of {C} x {G} values")
    if V is not None and not (isinstance(V, torch.Tensor) and V.is_cuda and V.dtype == torch.float64
                              and V.is_contiguous() and V.numel() == G and V.device == X.device):
        raise ValueError(f"V must be a contiguous float64 CUDA tensor of {G} values on X's device")
    pr = _noalloc_problem(F, n, lo, hi, beta, M, p, q)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    E = ctypes.c_double()
    _check(_lib.sbec_energy_noalloc(ctypes.byref(pr), _ptr(V), _ptr(X), ctypes.byref(E), stream),
           "sbec_energy_noalloc")
    return E.value


def energy_noalloc_raw(F, n, lo, hi, beta, M, X_ptr, p=0.0, q=0.0, V_ptr=0, stream=None):
    """sbec_energy_noalloc on raw addresses, without the checks of energy_noalloc;
    returns the status code (the energy is discarded).  For testing the entry
    point's own argument checks."""
    pr = _noalloc_problem(F, n, lo, hi, beta, M, p, q)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    E = ctypes.c_double()
    return int(_lib.sbec_energy_noalloc(ctypes.byref(pr), ctypes.c_void_p(V_ptr or None),
                                        ctypes.c_void_p(X_ptr), ctypes.byref(E), stream))


class SolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("retraction", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("rgbb_tol", ctypes.c_double), ("rgbb_maxit", ctypes.c_int),
                ("project_initial", ctypes.c_int), ("cg_chunk", ctypes.c_int), ("cuda_graphs", ctypes.c_int),
                ("refine_cg_fp32", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("grad_norm", ctypes.c_double),
                ("outer_iters", ctypes.c_longlong), ("inner_iters", ctypes.c_longlong),
                ("rgbb_iters", ctypes.c_longlong), ("n_grad", ctypes.c_longlong),
                ("n_energy", ctypes.c_longlong), ("n_hvp", ctypes.c_longlong),
                ("converged", ctypes.c_int)]


_lib.sbec_solve_defaults.argtypes = [ctypes.POINTER(SolveOpts)]
_lib.sbec_solve_defaults.restype = None
_lib.sbec_solve_workspace_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
_lib.sbec_solve_workspace_bytes.restype = _int
_lib.sbec_solve.argtypes = [_vp, _vp, ctypes.POINTER(SolveOpts), _vp, ctypes.c_size_t, ctypes.POINTER(Stats)]
_lib.sbec_solve.restype = _int
ARNT, RGBB = 0, 1


def _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, project=True, cg_chunk=None, graphs=None,
          refine_cg_fp32=None):
    """sbec_solve_opts from the library defaults and the given overrides (None keeps the
    default: 4 CG iterations per chunk, CUDA graphs on)."""
    o = SolveOpts()
    _lib.sbec_solve_defaults(ctypes.byref(o))
    o.method = ARNT if method == "arnt" else RGBB
    o.retraction, o.tol, o.maxit = int(retraction), float(tol), int(maxit)
    o.rgbb_tol, o.rgbb_maxit, o.project_initial = float(rgbb_tol), int(rgbb_maxit), int(bool(project))
    if cg_chunk is not None:
        o.cg_chunk = int(cg_chunk)
    if graphs is not None:
        o.cuda_graphs = int(bool(graphs))
    if refine_cg_fp32 is not None:
        o.refine_cg_fp32 = int(bool(refine_cg_fp32))
    return o


def _solve(self, X, method="arnt", retraction=1, tol=1e-8, maxit=10000, rgbb_tol=1e-2,
           rgbb_maxit=2000, project=True, workspace=None, cg_chunk=None, graphs=None):
    """Ground state from X (overwritten) by sbec_solve; returns the stats as a dict.
    Raises SbecError unless the tolerance was reached (status NOCONV included)."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, project, cg_chunk, graphs)
    nb = ctypes.c_size_t()
    _check(_lib.sbec_solve_workspace_bytes(self._h, ctypes.byref(nb)), "sbec_solve_workspace_bytes")
    if workspace is None:
        import torch
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    st = Stats()
    rc = _lib.sbec_solve(self._h, _ptr(X), ctypes.byref(o), _ptr(workspace), nb.value, ctypes.byref(st))
    out = {k: getattr(st, k) for k, _ in Stats._fields_}
    out["status"] = rc
    if rc not in (OK, ERR_NOCONV):
        _check(rc, "sbec_solve")
    return out


Handle.solve = _solve


_lib.sbec_solve_mixed_workspace_bytes.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]
_lib.sbec_solve_mixed_workspace_bytes.restype = _int
_lib.sbec_solve_mixed.argtypes = [_vp, _vp, _vp, ctypes.POINTER(SolveOpts), _dbl, _vp, ctypes.c_size_t,
                                  ctypes.POINTER(Stats), ctypes.POINTER(Stats)]
_lib.sbec_solve_mixed.restype = _int


def solve_mixed(h64, h32, X, tol=1e-8, tol_mixed=1e-3, method="arnt", retraction=1, maxit=10000,
                rgbb_tol=1e-2, rgbb_maxit=2000, workspace=None, cg_chunk=None, graphs=None, refine_cg_fp32=None):
    """Mixed-precision solve on h32 then FP64 refinement on h64 (sbec_solve_mixed).
    X: complex128 device tensor, overwritten.  refine_cg_fp32 (default on): the
    refinement's modified CG runs on h32.  Returns (stats_mixed, stats_fp64), dicts
    for single handles and lists of B dicts for batch handles."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, True, cg_chunk, graphs, refine_cg_fp32)
    nb = ctypes.c_size_t()
    _check(_lib.sbec_solve_mixed_workspace_bytes(h64._h, h32._h, ctypes.byref(nb)),
           "sbec_solve_mixed_workspace_bytes")
    if workspace is None:
        import torch
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    B = h64.B
    sm, sf = (Stats * B)(), (Stats * B)()
    rc = _lib.sbec_solve_mixed(h64._h, h32._h, _ptr(X), ctypes.byref(o), float(tol_mixed), _ptr(workspace),
                               nb.value, sm, sf)
    if rc not in (OK, ERR_NOCONV):
        _check(rc, "sbec_solve_mixed")
    a = [{k: getattr(sm[i], k) for k, _ in Stats._fields_} for i in range(B)]
    b = [dict({k: getattr(sf[i], k) for k, _ in Stats._fields_}, status=rc) for i in range(B)]
    return (a[0], b[0]) if B == 1 else (a, b)


_lib.sbec_prolongate.argtypes = [_vp, _vp, _vp, _vp]
_lib.sbec_prolongate.restype = _int
_lib.sbec_solve_cascadic.argtypes = [ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp), ctypes.POINTER(SolveOpts),
                                     _dbl, _vp, ctypes.c_size_t, ctypes.POINTER(Stats)]
_lib.sbec_solve_cascadic.restype = _int


def prolongate(hc, Xc, hf, Xf):
    """Cascadic prolongation of Xc (handle hc) to Xf (finer handle hf), sbec_prolongate."""
    _check(_lib.sbec_prolongate(hc._h, _ptr(Xc), hf._h, _ptr(Xf)), "sbec_prolongate")


def solve_cascadic(handles, states, tol=1e-8, tol_coarse=1e-5, method="arnt", retraction=1, maxit=10000,
                   rgbb_tol=1e-2, rgbb_maxit=2000, workspace=None, cg_chunk=None, graphs=None):
    """sbec_solve_cascadic over handles (coarse to fine); states[j] is level j's array
    (states[0] holds the initial data, the finest receives the ground state)."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, True, cg_chunk, graphs)
    nb = ctypes.c_size_t()
    _check(_lib.sbec_solve_workspace_bytes(handles[-1]._h, ctypes.byref(nb)), "sbec_solve_workspace_bytes")
    if workspace is None:
        import torch
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    hs = (_vp * len(handles))(*[h._h for h in handles])
    xs = (_vp * len(states))(*[_ptr(x) for x in states])
    st = Stats()
    rc = _lib.sbec_solve_cascadic(hs, len(handles), xs, ctypes.byref(o), float(tol_coarse), _ptr(workspace),
                                  nb.value, ctypes.byref(st))
    if rc not in (OK, ERR_NOCONV):
        _check(rc, "sbec_solve_cascadic")
    out = {k: getattr(st, k) for k, _ in Stats._fields_}
    out["status"] = rc
    return out


_lib.sbec_solve_cascadic_mixed.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp),
                                           ctypes.POINTER(SolveOpts), _dbl, _dbl, _vp, ctypes.c_size_t,
                                           ctypes.POINTER(Stats), ctypes.POINTER(Stats)]
_lib.sbec_solve_cascadic_mixed.restype = _int


def solve_cascadic_mixed(handles64, handles32, states, tol=1e-8, tol_coarse=1e-5, tol_mixed=1e-3, method="arnt",
                         retraction=1, maxit=10000, rgbb_tol=1e-2, rgbb_maxit=2000, workspace=None, cg_chunk=None,
                         graphs=None, refine_cg_fp32=None):
    """sbec_solve_cascadic_mixed: per level a mixed solve with FP64 refinement, coarse to
    fine; states[j] (complex128 device tensors) is level j's array.  Returns the
    (mixed, fp64) stats dicts of the finest level."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, True, cg_chunk, graphs, refine_cg_fp32)
    nb = ctypes.c_size_t()
    _check(_lib.sbec_solve_mixed_workspace_bytes(handles64[-1]._h, handles32[-1]._h, ctypes.byref(nb)),
           "sbec_solve_mixed_workspace_bytes")
    if workspace is None:
        import torch
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    h64 = (_vp * len(handles64))(*[h._h for h in handles64])
    h32 = (_vp * len(handles32))(*[h._h for h in handles32])
    xs = (_vp * len(states))(*[_ptr(x) for x in states])
    sm, sf = Stats(), Stats()
    rc = _lib.sbec_solve_cascadic_mixed(h64, h32, len(handles64), xs, ctypes.byref(o), float(tol_coarse),
                                        float(tol_mixed), _ptr(workspace), nb.value, ctypes.byref(sm),
                                        ctypes.byref(sf))
    if rc not in (OK, ERR_NOCONV):
        _check(rc, "sbec_solve_cascadic_mixed")
    a = {k: getattr(sm, k) for k, _ in Stats._fields_}
    b = dict({k: getattr(sf, k) for k, _ in Stats._fields_}, status=rc)
    return a, b


_lib.sbec_solve_graph.argtypes = [ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp), ctypes.POINTER(SolveOpts),
                                  ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t), ctypes.c_longlong,
                                  ctypes.POINTER(ctypes.POINTER(Stats))]
_lib.sbec_solve_graph.restype = _int


def solve_graph(handles, Xs, tol=1e-8, method="arnt", retraction=1, maxit=10000, rgbb_tol=1e-2, rgbb_maxit=2000,
                project=True, workspaces=None, loop_cap=0):
    """sbec_solve_graph: the solves of every instance of the given handles as one CUDA
    graph launch.  Xs[i] (device tensor of handle i) is overwritten.  Returns
    (status, [list of per-instance stats dicts per handle]); raises SbecError on a
    CUDA or argument error."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, project)
    nh = len(handles)
    sizes = []
    for h in handles:
        nb = ctypes.c_size_t()
        _check(_lib.sbec_solve_workspace_bytes(h._h, ctypes.byref(nb)), "sbec_solve_workspace_bytes")
        sizes.append(nb.value)
    if workspaces is None:
        import torch
        workspaces = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    stats = [(Stats * h.B)() for h in handles]
    hs = (_vp * nh)(*[h._h for h in handles])
    xs = (_vp * nh)(*[_ptr(x) for x in Xs])
    ws = (_vp * nh)(*[_ptr(x) for x in workspaces])
    nbs = (ctypes.c_size_t * nh)(*sizes)
    sp = (ctypes.POINTER(Stats) * nh)(*[ctypes.cast(st, ctypes.POINTER(Stats)) for st in stats])
    rc = _lib.sbec_solve_graph(hs, nh, xs, ctypes.byref(o), ws, nbs, int(loop_cap), sp)
    if rc not in (OK, ERR_NOCONV, ERR_TIMEOUT):
        _check(rc, "sbec_solve_graph")
    return rc, [[{k: getattr(st[i], k) for k, _ in Stats._fields_} for i in range(h.B)]
                for st, h in zip(stats, handles)]


_lib.sbec_solve_batch.argtypes = [_vp, _vp, ctypes.POINTER(SolveOpts), _vp, ctypes.c_size_t, ctypes.POINTER(Stats)]
_lib.sbec_solve_batch.restype = _int


def solve_batch(h, X, tol=1e-8, method="arnt", retraction=1, maxit=10000, rgbb_tol=1e-2, rgbb_maxit=2000,
                project=True, workspace=None, cg_chunk=None, graphs=None):
    """Lock-step ground-state solve of every instance of a batch handle (sbec_solve_batch).
    X: device tensor (B, C, ...), overwritten.  Returns a list of per-instance stats dicts."""
    o = _opts(method, retraction, tol, maxit, rgbb_tol, rgbb_maxit, project, cg_chunk, graphs)
    nb = ctypes.c_size_t()
    _check(_lib.sbec_solve_workspace_bytes(h._h, ctypes.byref(nb)), "sbec_solve_workspace_bytes")
    if workspace is None:
        import torch
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    st = (Stats * h.B)()
    rc = _lib.sbec_solve_batch(h._h, _ptr(X), ctypes.byref(o), _ptr(workspace), nb.value, st)
    if rc not in (OK, ERR_NOCONV):
        _check(rc, "sbec_solve_batch")
    return [dict({k: getattr(st[i], k) for k, _ in Stats._fields_}, status=rc) for i in range(h.B)]
