"""GB300 (sm_103a) DirectLiNGAM causal ordering -- thin Python binding.

Every function here only marshals arguments into the C ABI of
``include/lingam.h`` (``liblingam_gb300.so``); all arithmetic runs in the
library's CUDA kernels.  Importing this package never falls back to a CPU
path: if the shared library is missing or no CUDA device is present, the
calls raise.

Data arguments may be numpy arrays (host memory) or torch tensors (host or
CUDA).  A 2-D array of shape [n, d] (samples x variables, the paper's
[m, dim]) is passed as row-major when C-contiguous and as column-major when
its transpose is C-contiguous.  CUDA tensors are used in place on the
current torch stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "liblingam_gb300.so")

OK, ERR_ARG, ERR_NONFINITE, ERR_DEGENERATE, ERR_CUDA, ERR_OOM, ERR_TIMEOUT = range(7)
PREC = {"fp32": 0, "mixed": 1, "fp64": 2, "df": 3}
ROW_MAJOR, COL_MAJOR = 0, 1


class LingamError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lingam status {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("tie_scale", ctypes.c_double), ("conditional_rescore", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class Stats(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("pair_ms", ctypes.c_double),
                ("pair_launches", ctypes.c_int64), ("pair_units", ctypes.c_double),
                ("refined_steps", ctypes.c_int32), ("genuine_ties", ctypes.c_int32),
                ("candidates_max", ctypes.c_int32), ("graph_nodes", ctypes.c_int32),
                ("graph_build_ms", ctypes.c_double), ("fp64_candidates", ctypes.c_int32),
                ("df_candidates", ctypes.c_int32), ("cond_nodes", ctypes.c_int32),
                ("cond_bodies", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
                ("score_ms", ctypes.c_double),
                ("refine_ms", ctypes.c_double), ("regress_ms", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n_src", ctypes.c_int64), ("n", ctypes.c_int64),
                ("d", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("rows", ctypes.POINTER(ctypes.c_int32))]


class Tuning(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("p_max", ctypes.c_int32 * 8), ("tile", ctypes.c_int32 * 8),
                ("ctas_per_sm", ctypes.c_int32 * 8), ("p_probe", ctypes.c_int32 * 8),
                ("ms", ctypes.c_double * 8), ("n_probe", ctypes.c_int64)]

    def to_dict(self) -> dict:
        k = self.count
        return {"count": k, "precision": self.precision, "p_max": list(self.p_max[:k]),
                "tile": list(self.tile[:k]), "ctas_per_sm": list(self.ctas_per_sm[:k]),
                "p_probe": list(self.p_probe[:k]), "ms": list(self.ms[:k]),
                "n_probe": self.n_probe}

    @classmethod
    def from_dict(cls, t: dict) -> "Tuning":
        out = cls()
        out.count, out.precision, out.n_probe = t["count"], t["precision"], t.get("n_probe", 0)
        for name in ("p_max", "tile", "ctas_per_sm", "p_probe", "ms"):
            arr = getattr(out, name)
            for i, v in enumerate(t.get(name, [])[:8]):
                arr[i] = v
        return out


_lib = None

# name -> (restype, argtypes); every symbol declared in include/lingam.h
_P, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "lingam_create": (_I32, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(Opts)]),
    "lingam_destroy": (_I32, [_P]),
    "lingam_last_error": (ctypes.c_char_p, [_P]),
    "lingam_set_precision": (_I32, [_P, _I32]),
    "lingam_causal_order": (_I32, [_P, _P, _I64, _I64, _I64, _I32, _P, _P, _P]),
    "lingam_fit_adjacency": (_I32, [_P, _P, _I64, _I64, _I64, _I32, _P, _P, _I32, _P]),
    "varlingam_fit": (_I32, [_P, _P, _I64, _I64, _I64, _I32, _I32, _P, _P, _P, _P]),
    "lingam_causal_order_batch": (_I32, [_P, ctypes.POINTER(Instance), _I32, _P, _P, _P, _P]),
    "lingam_step_measures": (_I32, [_P, _P, _I64, _I64, _I64, _I32, _P, _P, _P, _P]),
    "lingam_get_stats": (_I32, [_P, ctypes.POINTER(Stats)]),
    "lingam_peak_probe": (_I32, [_P, _I32, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "lingam_step_scores_noalloc": (_I32, [_P, _I64, _I64, _I64, _P, _P]),
    "lingam_autotune": (_I32, [_P, _I64, _I64, _I32, ctypes.POINTER(Tuning)]),
    "lingam_total_effects": (_I32, [_P, _P, _I64, _P, _P, _I32, _P]),
    "lingam_prune_adjacency": (_I32, [_P, _P, _I64, _I64, _I64, _I32, _P, _D, _I32, _D, _P, _I32,
                                      _P]),
    "varlingam_total_effects": (_I32, [_P, _P, _P, _I64, _I32, _P, _P, _I32, _P]),
    "lingam_influence": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "lingam_bootstrap_edge_stats": (_I32, [_P, _P, _I32, _I64, _D, _P, _P, _P]),
    "lingam_set_tuning": (_I32, [_P, ctypes.POINTER(Tuning)]),
    "lingam_get_tuning": (_I32, [_P, _I32, ctypes.POINTER(Tuning)]),
    "lingam_pair_tile_info": (_I32, [_I32, ctypes.POINTER(_I32)]),
    "lingam_set_prior_knowledge": (_I32, [_P, ctypes.POINTER(ctypes.c_int8), _I64]),
    "lingam_set_input_gate": (_I32, [_P, _P, ctypes.c_double]),
    "lingam_set_shard": (_I32, [_P, _I32, _I32, _P, _P]),
    "lingam_shard_owner": (_I32, [_I64, _I64, _I64, _I32]),
}


def load(path: str = LIBPATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _torch():
    try:
        import torch
        return torch
    except Exception:      # torch is optional for host-only use
        return None


def _stream_of(arrs):
    torch = _torch()
    if torch is not None:
        for a in arrs:
            if isinstance(a, torch.Tensor) and a.is_cuda:
                return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return ctypes.c_void_p(0)


def _square_f64(A):
    """(pointer, size, keepalive) of a square FP64 matrix (host or CUDA)."""
    torch = _torch()
    if torch is not None and isinstance(A, torch.Tensor):
        if A.dtype != torch.float64 or A.dim() != 2 or A.shape[0] != A.shape[1]:
            raise TypeError("expected a square float64 tensor")
        A = A.contiguous()
        return ctypes.c_void_p(A.data_ptr()), A.shape[0], A
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("expected a square matrix")
    return ctypes.c_void_p(A.ctypes.data), A.shape[0], A


def _matrix(X, dtype):
    """(pointer, n, d, ld, layout, keepalive) of a 2-D array without copying
    device data; host data is converted to ``dtype`` contiguous if needed."""
    torch = _torch()
    if torch is not None and isinstance(X, torch.Tensor):
        tdt = torch.float64 if dtype == np.float64 else torch.float32
        if X.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {X.dtype}")
        if X.dim() != 2:
            raise ValueError("X must be 2-D [n, d]")
        n, d = X.shape
        if X.stride(1) == 1 and X.stride(0) >= d:
            return ctypes.c_void_p(X.data_ptr()), n, d, X.stride(0), ROW_MAJOR, X
        if X.stride(0) == 1 and X.stride(1) >= n:
            return ctypes.c_void_p(X.data_ptr()), n, d, X.stride(1), COL_MAJOR, X
        X = X.contiguous()
        return ctypes.c_void_p(X.data_ptr()), n, d, d, ROW_MAJOR, X
    A = np.asarray(X)
    if A.ndim != 2:
        raise ValueError("X must be 2-D [n, d]")
    if A.dtype != dtype:
        A = A.astype(dtype)
    n, d = A.shape
    if A.flags.c_contiguous:
        return ctypes.c_void_p(A.ctypes.data), n, d, d, ROW_MAJOR, A
    if A.flags.f_contiguous:
        return ctypes.c_void_p(A.ctypes.data), n, d, n, COL_MAJOR, A
    A = np.ascontiguousarray(A)
    return ctypes.c_void_p(A.ctypes.data), n, d, d, ROW_MAJOR, A


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Context:
    """A library context on one CUDA device (owns workspace and graphs)."""

    def __init__(self, device: int = 0, precision: str = "fp32", profile: bool = False,
                 tie_scale: float = 0.0, conditional_rescore: bool = False):
        lib = load()
        opts = Opts(PREC[precision], int(bool(profile)), float(tie_scale),
                    int(bool(conditional_rescore)))
        h = ctypes.c_void_p()
        code = lib.lingam_create(ctypes.byref(h), int(device), ctypes.byref(opts))
        if code != OK:
            raise LingamError(code, lib.lingam_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.precision = precision

    # -- plumbing --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lingam_destroy(self._h)
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

    def _check(self, code: int):
        if code != OK:
            raise LingamError(code, self._lib.lingam_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def set_precision(self, precision: str):
        self._check(self._lib.lingam_set_precision(self._h, PREC[precision]))
        self.precision = precision

    def _dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32

    def set_shard(self, rank: int, nranks: int, allreduce=None):
        """Compute only this rank's slice of the pair space (lingam_set_shard).

        ``allreduce(buf)`` receives a float64 numpy view of [partial M |
        partial E] (2 p values) after each step's scoring and must overwrite
        it with the sums over all ranks, identical on every rank."""
        if nranks <= 1:
            self._check(self._lib.lingam_set_shard(self._h, 0, 1, None, None))
            self._shard_cb = None
            return

        def trampoline(buf, count, user):
            try:
                allreduce(np.ctypeslib.as_array(buf, shape=(int(count),)))
                return 0
            except Exception:   # reported to the caller as a failed exchange
                return 1

        cb = _ALLREDUCE_FN(trampoline)
        self._check(self._lib.lingam_set_shard(self._h, int(rank), int(nranks),
                                               ctypes.cast(cb, ctypes.c_void_p), None))
        self._shard_cb = cb          # the library keeps calling it while set

    def set_input_gate(self, flag, timeout_s: float = 1.0):
        """Make lingam_causal_order / step_measures wait on the device until
        the uint32 ``flag`` (a CUDA tensor, or an integer device / mapped
        host address) is non-zero before reading their input; ``None``
        removes the gate.  A wait longer than ``timeout_s`` fails the call
        with ERR_TIMEOUT."""
        if flag is None:
            self._check(self._lib.lingam_set_input_gate(self._h, None, 0.0))
            self._gate = None
            return
        addr = flag.data_ptr() if hasattr(flag, "data_ptr") else int(flag)
        self._check(self._lib.lingam_set_input_gate(self._h, ctypes.c_void_p(addr),
                                                     float(timeout_s)))
        self._gate = flag           # keep the caller's buffer alive while set

    # -- the ABI ----------------------------------------------------------------
    def causal_order(self, X, scores: bool = False):
        p, n, d, ld, lay, keep = _matrix(X, self._dtype())
        order = np.empty(d, dtype=np.int32)
        sc = np.empty((d, d)) if scores else None
        code = self._lib.lingam_causal_order(self._h, p, n, d, ld, lay, _ptr(order),
                                             _ptr(sc) if sc is not None else None,
                                             _stream_of([keep]))
        self._check(code)
        return (order, sc) if scores else order

    def step_measures(self, X, bounds: bool = False):
        """(I [d, d], M [d]) of the first ordering step; with ``bounds`` also
        the per-entry bound on |I - I_exact| the library works with."""
        p, n, d, ld, lay, keep = _matrix(X, self._dtype())
        I = np.empty((d, d))
        M = np.empty(d)
        eps = np.empty((d, d)) if bounds else None
        self._check(self._lib.lingam_step_measures(self._h, p, n, d, ld, lay, _ptr(I), _ptr(M),
                                                   _ptr(eps) if bounds else None,
                                                   _stream_of([keep])))
        return (I, M, eps) if bounds else (I, M)

    def fit_adjacency(self, X, order, out=None):
        p, n, d, ld, lay, keep = _matrix(X, np.float32)
        order = np.ascontiguousarray(order, dtype=np.int32)
        torch = _torch()
        if out is not None and torch is not None and isinstance(out, torch.Tensor) and out.is_cuda:
            self._check(self._lib.lingam_fit_adjacency(self._h, p, n, d, ld, lay, _ptr(order),
                                                       ctypes.c_void_p(out.data_ptr()), 1,
                                                       _stream_of([keep, out])))
            return out
        B = np.empty((d, d))
        self._check(self._lib.lingam_fit_adjacency(self._h, p, n, d, ld, lay, _ptr(order),
                                                   _ptr(B), 0, _stream_of([keep])))
        return B

    def prune_adjacency(self, X, order, gamma: float = 1.0, n_lambda: int = 60,
                        eps: float = 1e-6):
        """Sparse adjacency: adaptive lasso + BIC of each variable on its
        predecessors in ``order`` (host float64 [d, d])."""
        p, n, d, ld, lay, keep = _matrix(X, np.float32)
        order = np.ascontiguousarray(order, dtype=np.int32)
        B = np.empty((d, d))
        self._check(self._lib.lingam_prune_adjacency(self._h, p, n, d, ld, lay, _ptr(order),
                                                     float(gamma), int(n_lambda), float(eps),
                                                     _ptr(B), 0, _stream_of([keep])))
        return B

    def varlingam_fit(self, Xt, lags: int = 1):
        """(order, B0, Btau[lags, d, d]) of VarLiNGAM on the series Xt [T, d]."""
        p, T, d, ld, lay, keep = _matrix(Xt, np.float32)
        order = np.empty(d, dtype=np.int32)
        B0 = np.empty((d, d))
        Bt = np.empty((lags, d, d))
        self._check(self._lib.varlingam_fit(self._h, p, T, d, ld, lay, int(lags), _ptr(order),
                                            _ptr(B0), _ptr(Bt), _stream_of([keep])))
        return order, B0, Bt

    # -- read-outs of the estimated graph (Sec. 4.2) -----------------------------
    def total_effects(self, B, order):
        """T = (I - B)^-1 (host float64 [d, d]); B must follow ``order``."""
        p, d, keep = _square_f64(B)
        order = np.ascontiguousarray(order, dtype=np.int32)
        T = np.empty((d, d))
        self._check(self._lib.lingam_total_effects(self._h, p, d, _ptr(order), _ptr(T), 0,
                                                   _stream_of([keep])))
        return T

    def varlingam_total_effects(self, B0, Btau, order):
        """Total effects over the time-unrolled nodes [x(t-lags) .. x(t)]."""
        p0, d, k0 = _square_f64(B0)
        Bt = np.ascontiguousarray(Btau, dtype=np.float64)
        if Bt.ndim != 3 or Bt.shape[1:] != (d, d):
            raise ValueError("Btau must be [lags, d, d]")
        lags = Bt.shape[0]
        order = np.ascontiguousarray(order, dtype=np.int32)
        q = (lags + 1) * d
        T = np.empty((q, q))
        self._check(self._lib.varlingam_total_effects(self._h, p0, _ptr(Bt), d, lags, _ptr(order),
                                                      _ptr(T), 0, _stream_of([k0])))
        return T

    def influence(self, T):
        """(exert, receive, exert_rank, receive_rank) of every node."""
        p, q, keep = _square_f64(T)
        ex, rc = np.empty(q), np.empty(q)
        rex, rrc = np.empty(q, dtype=np.int32), np.empty(q, dtype=np.int32)
        self._check(self._lib.lingam_influence(self._h, p, q, _ptr(ex), _ptr(rc), _ptr(rex),
                                               _ptr(rrc), _stream_of([keep])))
        return ex, rc, rex, rrc

    def bootstrap_edge_stats(self, Bs, threshold: float = 0.0):
        """(prob, mean) of the edges over a list of [d, d] adjacency matrices."""
        keep = [_square_f64(B) for B in Bs]
        if not keep:
            raise ValueError("need at least one matrix")
        d = keep[0][1]
        if any(k[1] != d for k in keep):
            raise ValueError("all matrices must be d x d")
        ptrs = (ctypes.c_void_p * len(keep))(*[k[0].value for k in keep])
        prob, mean = np.empty((d, d)), np.empty((d, d))
        self._check(self._lib.lingam_bootstrap_edge_stats(
            self._h, ptrs, len(keep), d, float(threshold), _ptr(prob), _ptr(mean),
            _stream_of([k[2] for k in keep])))
        return prob, mean

    def causal_order_batch(self, instances, adjacency: bool = False):
        """instances: list of (X [n_src, d] float32, rows int32[n] or None).
        Returns the list of orders (and adjacency matrices when asked)."""
        keep = []
        arr = (Instance * len(instances))()
        orders = []
        Bs = []
        for k, (X, rows) in enumerate(instances):
            p, n_src, d, ld, lay, kx = _matrix(X, np.float32)
            if lay != ROW_MAJOR:
                raise ValueError("batch instances must be row-major")
            keep.append(kx)
            if rows is not None:
                r = np.ascontiguousarray(rows, dtype=np.int32)
                keep.append(r)
                arr[k] = Instance(p, n_src, r.size, d, ld,
                                  r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
            else:
                arr[k] = Instance(p, n_src, n_src, d, ld, None)
            orders.append(np.empty(d, dtype=np.int32))
            Bs.append(np.empty((d, d)) if adjacency else None)
        optr = (ctypes.c_void_p * len(instances))(*[o.ctypes.data for o in orders])
        bptr = (ctypes.c_void_p * len(instances))(*[b.ctypes.data for b in Bs]) if adjacency else None
        failed = ctypes.c_int32(-1)
        code = self._lib.lingam_causal_order_batch(self._h, arr, len(instances), optr, bptr,
                                                   ctypes.byref(failed), _stream_of(keep))
        self._check(code)
        return (orders, Bs) if adjacency else orders

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.lingam_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_ if k != "reserved"}

    def autotune(self, n: int, d: int, cache: str | None = None, instances: int = 1) -> dict:
        """Tile shapes and split schedules of the FP32 pair kernel for problems
        of n samples and up to d variables (``instances`` of them per batch),
        in the context's form.  With ``cache`` (a JSON file) a table saved for
        the same GPU model, form and sizes is installed instead of
        re-measuring, and a new one is saved."""
        import json
        key = None
        if cache:
            torch = _torch()
            dev = torch.cuda.get_device_name(0) if torch and torch.cuda.is_available() else "gpu"
            key = f"{dev}|{self.precision}|n={int(n)}|d={int(d)}|k={int(instances)}"
            try:
                with open(cache) as f:
                    saved = json.load(f)
            except (OSError, ValueError):
                saved = {}
            if key in saved:
                t = Tuning.from_dict(saved[key])
                self._check(self._lib.lingam_set_tuning(self._h, ctypes.byref(t)))
                return saved[key]
        t = Tuning()
        self._check(self._lib.lingam_autotune(self._h, int(n), int(d), int(instances),
                                              ctypes.byref(t)))
        out = t.to_dict()
        if cache:
            try:
                with open(cache) as f:
                    saved = json.load(f)
            except (OSError, ValueError):
                saved = {}
            saved[key] = out
            with open(cache, "w") as f:
                json.dump(saved, f, indent=1)
        return out

    def tuning(self, precision: str | None = None) -> dict:
        t = Tuning()
        self._check(self._lib.lingam_get_tuning(self._h, PREC[precision or self.precision],
                                                ctypes.byref(t)))
        return t.to_dict()

    def set_tuning(self, table: dict):
        t = Tuning.from_dict(table)
        self._check(self._lib.lingam_set_tuning(self._h, ctypes.byref(t)))

    def set_prior_knowledge(self, prior=None):
        """Ancestry knowledge for later orderings: [d, d] with prior[i, j] = 1
        if x_j is known to be an ancestor of x_i, 0 if known not to be, -1
        unknown; None clears it."""
        if prior is None:
            self._check(self._lib.lingam_set_prior_knowledge(self._h, None, 0))
            return
        pk = np.ascontiguousarray(np.asarray(prior), dtype=np.int8)
        if pk.ndim != 2 or pk.shape[0] != pk.shape[1]:
            raise LingamError(1, "prior knowledge must be a square [d, d] matrix")
        self._check(self._lib.lingam_set_prior_knowledge(
            self._h, pk.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), pk.shape[0]))

    def peak_probe(self, which: int):
        """(ops per second, SM MHz) of unit `which`: 0 FP32 FMA flop/s,
        1 MUFU ex2, 2 MUFU lg2, 3 FP64 FMA flop/s."""
        r, mhz = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lingam_peak_probe(self._h, int(which), ctypes.byref(r),
                                                ctypes.byref(mhz)))
        return r.value, mhz.value


# Module-level names mirroring the C ABI (same names, same argument order
# after the context).
def lingam_create(device: int = 0, precision: str = "fp32", profile: bool = False) -> Context:
    return Context(device, precision, profile)


def lingam_destroy(ctx: Context):
    ctx.close()


def lingam_causal_order(ctx: Context, X, scores: bool = False):
    return ctx.causal_order(X, scores)


def lingam_fit_adjacency(ctx: Context, X, order):
    return ctx.fit_adjacency(X, order)


def varlingam_fit(ctx: Context, Xt, lags: int = 1):
    return ctx.varlingam_fit(Xt, lags)


def lingam_causal_order_batch(ctx: Context, instances, adjacency: bool = False):
    return ctx.causal_order_batch(instances, adjacency)


def lingam_step_measures(ctx: Context, X):
    return ctx.step_measures(X)


PAIR_TILES = 33
_TILE_KEYS = ("wi", "wj", "wgi", "wgj", "stages", "groups", "fold", "packed", "sub")


_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                 ctypes.c_void_p)


def shard_owner(i: int, j: int, p: int, nranks: int) -> int:
    """Owner rank of the pairs (i, j) and (j, i) at a step with p remaining
    variables (lingam_shard_owner; no GPU needed)."""
    return int(load().lingam_shard_owner(int(i), int(j), int(p), int(nranks)))


def lingam_pair_tile_info(tile: int) -> dict:
    """Shape of pair-kernel tile configuration `tile` (no GPU needed): pairs
    per warp (wi x wj), warps (wgi x wgj), TMA stages, groups of 4 samples per
    lane and iteration (one lg2 per 4 x groups samples in the fast form),
    chunks between compensated folds, paired-FP32 arithmetic, chunks per
    ring stage of the streamlined block (0: the original block)."""
    out = (ctypes.c_int32 * 9)()
    st = load().lingam_pair_tile_info(int(tile), out)
    if st != 0:
        raise LingamError(st, f"lingam_pair_tile_info({tile}): no such tile configuration")
    return dict(zip(_TILE_KEYS, list(out)))
