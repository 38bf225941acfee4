"""Thin ctypes binding of the C ABI in include/convex_barrier.h (argument marshalling only).

Every step of the method runs in the CUDA library; this module only converts arrays to pointers.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA). Loading fails loudly
when the library has not been built: there is no CPU fallback.

  Context                 as_init .. as_destroy: as_step, sp_step, bound, backward (fixed bounds or
                          through interval propagation), get/set_state, export/import_state
  intermediate_bounds     as_intermediate_bounds (App. E)
  bab, bab_default_options  as_bab: branch and bound with stratified bounding (Sec. 6.2)
  ibp_noalloc             as_ibp_noalloc
  gemm_bf16               as_gemm_bf16
  default_options(input_l2=1, precision=16, ...)  the ellipsoid input set, the BF16 form
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libconvex_barrier.so")

AS_OK, AS_ERR_ARG, AS_ERR_SHAPE, AS_ERR_CUDA, AS_ERR_OOM, AS_ERR_NUMERIC, AS_ERR_TIMEOUT, AS_ERR_STATE, \
    AS_ERR_SCRATCH = range(9)
NOALLOC_SCRATCH_FLOATS = 1 << 22
LINEAR, CONV2D = 0, 1
MAX_LAYERS, MAX_CUTS = 10, 8

(ST_ALPHA, ST_BETA0, ST_BETA1, ST_SLOT_BETA, ST_XSNAP, ST_ZSNAP, ST_ITER, ST_LHAT, ST_UHAT, ST_XSTAR,
 ST_ZSTAR, ST_LAMBDA, ST_KAPPA, ST_ADAM, ST_SLOT_ADAM, ST_SP_X, ST_SP_Z, ST_SP_STATS, ST_SP_CAPS,
 ST_LO, ST_HI, ST_SP_SEL) = range(22)

EXPORTS = ["as_default_options", "as_init", "as_reset", "as_step", "sp_step", "as_bound",
           "as_bound_backward", "as_state_size", "as_get_state", "as_set_state", "as_launch_count",
           "as_kernel_times", "as_destroy", "as_last_error", "as_ibp_noalloc", "as_gemm_bf16",
           "as_team_targets", "as_intermediate_bounds", "as_bab", "as_bab_default_options", "as_bound_backward_ibp",
           "as_export_size", "as_export_state", "as_import_state"]
KERNELS = ["as_colA", "as_rowB", "reduce", "sp_colA", "sp_rowB", "sp_colC", "spi_row", "spi_col", "tc_col",
           "tc_row", "slot_sums", "ball_x0", "batch", "sp_start", "counter"]


class Layer(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("in_c", ct.c_int), ("in_h", ct.c_int), ("in_w", ct.c_int),
                ("out_c", ct.c_int), ("out_h", ct.c_int), ("out_w", ct.c_int), ("kh", ct.c_int),
                ("kw", ct.c_int), ("stride", ct.c_int), ("pad", ct.c_int),
                ("W", ct.c_void_p), ("b", ct.c_void_p)]


class Net(ct.Structure):
    _fields_ = [("n_layers", ct.c_int), ("layers", ct.POINTER(Layer))]


class Options(ct.Structure):
    _fields_ = [("bigm_iters", ct.c_int), ("as_iters", ct.c_int),
                ("bigm_lr0", ct.c_double), ("bigm_lr1", ct.c_double),
                ("as_lr0", ct.c_double), ("as_lr1", ct.c_double),
                ("omega", ct.c_int), ("vars_per_add", ct.c_int), ("max_cuts", ct.c_int),
                ("adam_b1", ct.c_double), ("adam_b2", ct.c_double), ("adam_eps", ct.c_double),
                ("sp_gamma0", ct.c_double), ("sp_c_alpha", ct.c_double), ("sp_c_beta", ct.c_double),
                ("sp_init_steps", ct.c_int), ("sp_init_lr0", ct.c_double), ("sp_init_lr1", ct.c_double),
                ("track_best", ct.c_int), ("graph_chunk", ct.c_int), ("profile", ct.c_int),
                ("autotune", ct.c_int), ("precision", ct.c_int), ("input_l2", ct.c_int)]


class BabOptions(ct.Structure):
    _fields_ = [("loose", Options), ("tight", Options), ("stratify", ct.c_int), ("cost_ratio", ct.c_double),
                ("ema_weight", ct.c_double), ("batch", ct.c_int), ("max_domains", ct.c_longlong),
                ("time_limit", ct.c_double), ("warm_start", ct.c_int), ("leaf_rebounds", ct.c_int),
                ("root_intermediate", ct.c_int), ("intermediate", Options)]


class BabResult(ct.Structure):
    _fields_ = [("status", ct.c_int), ("lower", ct.c_double), ("upper", ct.c_double), ("bounded", ct.c_longlong),
                ("hard_bounded", ct.c_longlong), ("batches", ct.c_longlong), ("max_depth", ct.c_longlong),
                ("frontier", ct.c_longlong), ("seconds", ct.c_double), ("cost_ratio", ct.c_double)]


BAB_STATUS = {0: "unknown", 1: "verified", 2: "falsified"}

_lib = None


def lib() -> ct.CDLL:
    """The loaded library; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing")
        L = ct.CDLL(LIB_PATH)
        L.as_default_options.argtypes = [ct.POINTER(Options)]
        L.as_default_options.restype = None
        L.as_init.argtypes = [ct.POINTER(ct.c_void_p), ct.POINTER(Net), ct.c_int] + [ct.c_void_p] * 7 + \
            [ct.POINTER(Options), ct.c_void_p]
        L.as_init.restype = ct.c_int
        L.as_reset.argtypes = [ct.c_void_p] + [ct.c_void_p] * 7
        L.as_kernel_times.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong)]
        L.as_step.argtypes = [ct.c_void_p, ct.c_int]
        L.sp_step.argtypes = [ct.c_void_p, ct.c_int]
        L.as_bound.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p]
        L.as_bound_backward_ibp.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                            ct.c_void_p]
        L.as_bound_backward_ibp.restype = ct.c_int
        L.as_bound_backward.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                        ct.c_void_p]
        L.as_state_size.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_longlong)]
        L.as_get_state.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
        L.as_set_state.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
        L.as_launch_count.argtypes = [ct.c_void_p]
        L.as_launch_count.restype = ct.c_longlong
        L.as_destroy.argtypes = [ct.c_void_p]
        L.as_destroy.restype = None
        L.as_last_error.argtypes = [ct.c_void_p]
        L.as_last_error.restype = ct.c_char_p
        L.as_ibp_noalloc.argtypes = [ct.POINTER(Net), ct.c_int] + [ct.c_void_p] * 6
        L.as_ibp_noalloc.restype = ct.c_int
        L.as_gemm_bf16.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int,
                                   ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]
        L.as_gemm_bf16.restype = ct.c_int
        L.as_team_targets.argtypes = [ct.c_void_p, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]
        L.as_team_targets.restype = ct.c_int
        L.as_intermediate_bounds.argtypes = [ct.POINTER(Net), ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                             ct.POINTER(Options), ct.c_longlong, ct.c_void_p, ct.c_void_p,
                                             ct.c_void_p]
        L.as_intermediate_bounds.restype = ct.c_int
        L.as_export_size.argtypes = [ct.c_void_p, ct.POINTER(ct.c_longlong)]
        L.as_export_size.restype = ct.c_int
        L.as_export_state.argtypes = [ct.c_void_p, ct.c_void_p]
        L.as_export_state.restype = ct.c_int
        L.as_import_state.argtypes = [ct.c_void_p, ct.c_void_p]
        L.as_import_state.restype = ct.c_int
        L.as_bab_default_options.argtypes = [ct.POINTER(BabOptions)]
        L.as_bab_default_options.restype = None
        L.as_bab.argtypes = [ct.POINTER(Net), ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(BabOptions),
                             ct.POINTER(BabResult), ct.c_void_p, ct.c_void_p]
        L.as_bab.restype = ct.c_int
        _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    lib().as_default_options(ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class CBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"convex-barrier error {code}: {msg}")
        self.code = code


def _ptr(a):
    """Pointer of a numpy array or torch tensor (contiguous), or None."""
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
    raise TypeError(type(a))


def _snapshot(a):
    """A float32 copy of an array or tensor's current values (host numpy, or a tensor on its device)."""
    if isinstance(a, np.ndarray):
        return np.array(a, np.float32, copy=True)
    return a.detach().to(dtype=a.dtype).clone()


def _layer_struct(L: dict, keep: list) -> Layer:
    W = np.ascontiguousarray(L["W"], np.float32) if isinstance(L["W"], np.ndarray) else L["W"]
    b = np.ascontiguousarray(L["b"], np.float32) if isinstance(L["b"], np.ndarray) else L["b"]
    keep += [W, b]
    s = Layer()
    if L["kind"] == "linear":
        s.kind, s.in_c, s.out_c = LINEAR, L["n_in"], L["n_out"]
        s.in_h = s.in_w = s.out_h = s.out_w = s.kh = s.kw = s.stride = 1
        s.pad = 0
    else:
        s.kind = CONV2D
        s.in_c, s.in_h, s.in_w = L["in_shape"]
        s.out_c, s.out_h, s.out_w = L["out_shape"]
        s.kh, s.kw, s.stride, s.pad = L["kh"], L["kw"], L["stride"], L["pad"]
    s.W, s.b = _ptr(W), _ptr(b)
    return s


class Context:
    """One solver context (as_ctx) over S subproblems."""

    def __init__(self, net: list, lo, hi, C=None, lhat=None, uhat=None, splits=None, caps=None,
                 options: Options | None = None, stream: int = 0):
        L = lib()
        keep = []
        layers = (Layer * len(net))(*[_layer_struct(x, keep) for x in net])
        self._net = Net(len(net), layers)
        self._keep = keep + [layers]
        conv = lambda a, dt: (np.ascontiguousarray(a, dt) if isinstance(a, np.ndarray) else a)
        lo, hi = conv(lo, np.float32), conv(hi, np.float32)
        C = conv(C, np.float32)
        lhat, uhat = conv(lhat, np.float32), conv(uhat, np.float32)
        splits = conv(splits, np.int8)
        caps = conv(caps, np.int32)
        self._keep += [lo, hi, C, lhat, uhat, splits, caps]
        self.S = int(lo.shape[0])
        self.options = options if options is not None else default_options()
        h = ct.c_void_p()
        r = L.as_init(ct.byref(h), ct.byref(self._net), self.S, _ptr(lo), _ptr(hi), _ptr(C), _ptr(lhat),
                      _ptr(uhat), _ptr(splits), _ptr(caps), ct.byref(self.options), ct.c_void_p(stream))
        self.h = h
        if r != AS_OK:
            msg = L.as_last_error(h).decode() if h.value else ""
            if h.value:
                L.as_destroy(h)
            self.h = ct.c_void_p()
            raise CBError(r, msg)
        self.n_layers = len(net)
        # the values the context was built on (weights) and is bounding (box): the differentiable
        # bound (autograd.py) refuses tensors that differ from them
        self._weights = [_snapshot(x[k]) for x in net for k in ("W", "b")]
        self._box = (_snapshot(lo), _snapshot(hi))
        self.widths = [net[0]["n_in"]] + [x["n_out"] for x in net[:-1]]
        self.NT = sum(self.widths)
        self.NH = self.NT - self.widths[0]
        self.cap = max(1, self.options.max_cuts)

    def _check(self, r):
        if r != AS_OK:
            raise CBError(r, lib().as_last_error(self.h).decode())

    def reset(self, lo, hi, C=None, lhat=None, uhat=None, splits=None, caps=None):
        """New batch on the same context (pointers: numpy host arrays or torch tensors)."""
        conv = lambda a, dt: (np.ascontiguousarray(a, dt) if isinstance(a, np.ndarray) else a)
        args = [conv(lo, np.float32), conv(hi, np.float32), conv(C, np.float32), conv(lhat, np.float32),
                conv(uhat, np.float32), conv(splits, np.int8), conv(caps, np.int32)]
        self._reset_keep = args
        self._check(lib().as_reset(self.h, *[_ptr(a) for a in args]))
        self._box = (_snapshot(args[0]), _snapshot(args[1]))

    def holds(self, lo, hi, params) -> str | None:
        """None when lo, hi and params = [W_1, b_1, ..., W_n, b_n] hold the values this context
        bounds (its box since creation or the last reset, its weights since creation); else which
        of them differs."""
        import torch

        def same(t, ref):
            t = t.detach()
            r = torch.as_tensor(ref).to(device=t.device, dtype=torch.float32)
            return t.shape == r.shape and bool(torch.equal(t.to(torch.float32), r))

        if len(params) != len(self._weights):
            return f"{len(params)} weight tensors given, the net has {len(self._weights)}"
        for q, (t, ref) in enumerate(zip(params, self._weights)):
            if not same(t, ref):
                return f"{'W' if q % 2 == 0 else 'b'}_{q // 2 + 1} differs from the weights the context was built on"
        if not same(lo, self._box[0]) or not same(hi, self._box[1]):
            return "the box differs from the one the context is bounding"
        return None

    def team_targets(self) -> tuple:
        """(row, col) team-size targets of the float32 passes: defaults or as_options.autotune's."""
        r, c = ct.c_longlong(), ct.c_longlong()
        self._check(lib().as_team_targets(self.h, ct.byref(r), ct.byref(c)))
        return r.value, c.value

    def kernel_times(self) -> dict:
        """{kernel name: (total ms, launches)} with options.profile = 1."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms, n = ct.c_double(), ct.c_longlong()
            self._check(lib().as_kernel_times(self.h, k, ct.byref(ms), ct.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def as_step(self, n: int):
        self._check(lib().as_step(self.h, n))

    def sp_step(self, n: int):
        self._check(lib().sp_step(self.h, n))

    def bound(self, precision: int = 64, best: bool = False):
        out = np.zeros(self.S, np.float64)
        bb = np.zeros(self.S, np.float64) if best else None
        self._check(lib().as_bound(self.h, precision, _ptr(out), _ptr(bb)))
        return (out, bb) if best else out

    def bound_into(self, precision: int, out, best=None):
        self._check(lib().as_bound(self.h, precision, _ptr(out), _ptr(best)))

    def backward(self, grad_bound, dW: list, db: list, dlo=None, dhi=None, through_bounds: bool = False):
        """as_bound_backward (intermediate bounds held fixed), or as_bound_backward_ibp with
        through_bounds (differentiated through the interval propagation that produced them)."""
        g = np.ascontiguousarray(grad_bound, np.float64) if isinstance(grad_bound, np.ndarray) else grad_bound
        n = self.n_layers
        pw = (ct.c_void_p * n)(*[_ptr(x) for x in dW]) if dW is not None else None
        pb = (ct.c_void_p * n)(*[_ptr(x) for x in db]) if db is not None else None
        fn = lib().as_bound_backward_ibp if through_bounds else lib().as_bound_backward
        self._check(fn(self.h, _ptr(g), ct.cast(pw, ct.c_void_p) if pw else None,
                       ct.cast(pb, ct.c_void_p) if pb else None, _ptr(dlo), _ptr(dhi)))

    def export_state(self) -> np.ndarray:
        """as_export_state: the whole iteration state as one byte blob (host)."""
        n = ct.c_longlong()
        self._check(lib().as_export_size(self.h, ct.byref(n)))
        out = np.zeros(n.value, np.uint8)
        self._check(lib().as_export_state(self.h, _ptr(out)))
        return out

    def import_state(self, blob: np.ndarray):
        """as_import_state: continue from a blob of export_state (same net, batch size, max_cuts)."""
        self._check(lib().as_import_state(self.h, _ptr(np.ascontiguousarray(blob, np.uint8))))

    def state_size(self, which: int) -> int:
        n = ct.c_longlong()
        self._check(lib().as_state_size(self.h, which, ct.byref(n)))
        return n.value

    def get_state(self, which: int, dtype=np.float32) -> np.ndarray:
        nb = self.state_size(which)
        out = np.zeros(nb // np.dtype(dtype).itemsize, dtype)
        self._check(lib().as_get_state(self.h, which, _ptr(out)))
        return out

    def set_state(self, which: int, arr):
        a = np.ascontiguousarray(arr)
        if a.nbytes != self.state_size(which):
            raise ValueError(f"state {which}: {a.nbytes} bytes, expected {self.state_size(which)}")
        self._check(lib().as_set_state(self.h, which, _ptr(a)))

    def launch_count(self) -> int:
        return lib().as_launch_count(self.h)

    def close(self):
        if self.h is not None and self.h.value:
            lib().as_destroy(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ibp_noalloc(net: list, lo, hi, lhat_out, uhat_out, splits=None, stream: int = 0) -> int:
    """as_ibp_noalloc: interval bounds with no allocation inside the call. Every array must be a
    CUDA tensor (weights and biases of `net` included); returns the status code."""
    keep = []
    layers = (Layer * len(net))(*[_layer_struct(x, keep) for x in net])
    n = Net(len(net), layers)
    return lib().as_ibp_noalloc(ct.byref(n), int(lo.shape[0]), _ptr(lo), _ptr(hi), _ptr(splits),
                                _ptr(lhat_out), _ptr(uhat_out), ct.c_void_p(stream))


def intermediate_bounds(net: list, lo, hi, splits=None, options: Options | None = None, max_batch: int = 0,
                        stream: int = 0):
    """as_intermediate_bounds: pre-activation bounds [S][NH] (lhat, uhat) of every hidden layer,
    layers 2 .. n-1 tightened by batched Big-M / Active Set solves over sub-networks. Arrays are
    numpy (host) or torch tensors; numpy outputs are returned."""
    keep = []
    layers = (Layer * len(net))(*[_layer_struct(x, keep) for x in net])
    n = Net(len(net), layers)
    conv = lambda a, dt: (np.ascontiguousarray(a, dt) if isinstance(a, np.ndarray) else a)
    lo, hi, splits = conv(lo, np.float32), conv(hi, np.float32), conv(splits, np.int8)
    S = int(lo.shape[0])
    NH = sum(x["n_out"] for x in net[:-1])
    lhat = np.empty((S, NH), np.float32)
    uhat = np.empty((S, NH), np.float32)
    opt = options if options is not None else default_options()
    r = lib().as_intermediate_bounds(ct.byref(n), S, _ptr(lo), _ptr(hi), _ptr(splits), ct.byref(opt),
                                     int(max_batch), _ptr(lhat), _ptr(uhat), ct.c_void_p(stream))
    if r != AS_OK:
        raise CBError(r, "as_intermediate_bounds")
    return lhat, uhat


def bab_default_options(loose=None, tight=None, intermediate=None, **kw) -> BabOptions:
    """as_bab_default_options, then the given fields (loose / tight / intermediate: dicts of
    as_options fields applied on top of their defaults)."""
    o = BabOptions()
    lib().as_bab_default_options(ct.byref(o))
    for name, d in (("loose", loose), ("tight", tight), ("intermediate", intermediate)):
        for k, v in (d or {}).items():
            setattr(getattr(o, name), k, v)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def bab(net: list, lo, hi, crow=None, options: BabOptions | None = None, stream: int = 0) -> dict:
    """as_bab: branch and bound with stratified bounding for crow . f(x) > 0 over the box [lo, hi]
    (host arrays); returns the result fields, the status as a word and the point of `upper`."""
    keep = []
    layers = (Layer * len(net))(*[_layer_struct(x, keep) for x in net])
    n = Net(len(net), layers)
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    c = None if crow is None else np.ascontiguousarray(crow, np.float32)
    opt = options if options is not None else bab_default_options()
    res = BabResult()
    x = np.full(lo.shape, np.nan, np.float32)
    r = lib().as_bab(ct.byref(n), _ptr(lo), _ptr(hi), _ptr(c), ct.byref(opt), ct.byref(res), _ptr(x),
                     ct.c_void_p(stream))
    if r != AS_OK:
        raise CBError(r, "as_bab")
    out = {f: getattr(res, f) for f, _ in BabResult._fields_}
    out["status"] = BAB_STATUS[res.status]
    out["x"] = None if np.isnan(x).any() else x
    return out


def gemm_bf16(A, B, D, bn: int = 128, stream: int = 0) -> int:
    """as_gemm_bf16: D = A . B^T for CUDA tensors A [M][K], B [N][K] (torch.bfloat16) and D [M][N]
    (float32), each with contiguous rows (row strides may exceed the row length); returns the
    status code."""
    M, K = A.shape
    N = B.shape[0]
    for t in (A, B, D):
        if t.stride(1) != 1:
            raise ValueError("rows must be contiguous")
    return lib().as_gemm_bf16(ct.c_void_p(A.data_ptr()), A.stride(0), ct.c_void_p(B.data_ptr()), B.stride(0),
                              ct.c_void_p(D.data_ptr()), D.stride(0), M, N, K, bn, ct.c_void_p(stream))


def context_for(prob: dict, options: Options | None = None, bounds=None, stream: int = 0, **kw) -> Context:
    """A Context for a synthetic problem dict (see synth.problem)."""
    lh = uh = None
    if bounds is not None:
        lh, uh = bounds
    return Context(prob["net"], prob["lo"], prob["hi"], prob["C"], lh, uh, prob.get("splits"),
                   prob.get("caps"), options, stream, **kw)
