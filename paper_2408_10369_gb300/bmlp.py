"""Python binding of the C ABI in ``include/bmlp.h`` (argument marshalling only).

Every function here forwards to the CUDA library ``_build/libbmlp.so``; there
is no Python or CPU implementation of any step. If the library cannot be
loaded, every call raises ``RuntimeError``.

Arrays may be ``torch.Tensor`` (device or host memory) or ``numpy.ndarray``
(host memory); their data pointers are passed through unchanged. The CUDA
stream is the caller's ``stream`` argument, else torch's current stream for
the context's device.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "bmlp.h")

BMLP_OK = 0
BMLP_ERR_INVALID_ARG = 1
BMLP_ERR_OOM = 2
BMLP_ERR_CUDA = 3
BMLP_ERR_TIMEOUT = 4
BMLP_ERR_NOT_CONVERGED = 5
BMLP_ERR_UNSUPPORTED = 6
BMLP_ERR_BUDGET = 7

BMLP_FMT_U8 = 0
BMLP_FMT_PACKED64 = 1
BMLP_FMT_I8 = 2
BMLP_FMT_E4M3 = 3

BMLP_AUTO = 0
BMLP_RMS_TC = 1
BMLP_RMS_PACKED = 2
BMLP_SMP_TC = 3
BMLP_SMP_PACKED = 4

BMLP_LOOP_HOST = 0
BMLP_LOOP_GRAPH = 1

VARIANTS = {"auto": BMLP_AUTO, "rms_tc": BMLP_RMS_TC, "rms_packed": BMLP_RMS_PACKED,
            "smp_tc": BMLP_SMP_TC, "smp_packed": BMLP_SMP_PACKED}
VARIANT_LIST = ["auto", "rms_tc", "rms_packed", "smp_tc", "smp_packed"]   # index = bmlp_variant

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NOT_CONVERGED", 6: "UNSUPPORTED",
           7: "BUDGET"}


class bmlp_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("reflexive", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("loop", ctypes.c_int32), ("profile", ctypes.c_int32), ("tc_only", ctypes.c_int32),
                ("timeout_ns", ctypes.c_uint64), ("budget_ns", ctypes.c_uint64), ("e4m3_only", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class bmlp_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("variant", ctypes.c_int32), ("product_launches", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("n_pad", ctypes.c_int64), ("product_ms", ctypes.c_double),
                ("issued_ops", ctypes.c_double), ("e2m1_products", ctypes.c_int32), ("frontier_squarings", ctypes.c_int32),
                ("sparse_squarings", ctypes.c_int32), ("sliced_closures", ctypes.c_int32), ("sparse_ms", ctypes.c_double),
                ("sparse_words", ctypes.c_double), ("host_syncs", ctypes.c_int32), ("cluster_frontiers", ctypes.c_int32),
                ("thin_squarings", ctypes.c_int32), ("table_squarings", ctypes.c_int32)]


class bmlp_problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("fmt", ctypes.c_int32), ("reflexive", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("n", ctypes.c_int64), ("R1", ctypes.c_void_p),
                ("R2", ctypes.c_void_p), ("out", ctypes.c_void_p)]


BMLP_PROBLEM_CLOSURE = 0
BMLP_PROBLEM_COMPOSE = 1

BMLP_NFEAT = 16
BMLP_NVAR = 4
BMLP_MLP_PARAMS = 5508


class bmlp_train_cfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("weight_decay", ctypes.c_float), ("seed", ctypes.c_uint64)]


class BmlpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("bmlp status %d (%s): %s" % (status, _STATUS.get(status, "?"), msg))
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return os.path.join(HERE, "_build", "libbmlp.so")


def lib():
    """Load (building first if needed) the CUDA library. Raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            try:
                path = _build.build()
            except Exception as e:  # no nvcc, compile error: fail loudly
                raise RuntimeError("the bmlp CUDA library is not available: %s" % e) from e
            L = ctypes.CDLL(path)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.bmlp_ctx_create.argtypes = [ctypes.POINTER(vp), i32]
            L.bmlp_ctx_destroy.argtypes = [vp]
            L.bmlp_last_error.argtypes = [vp]
            L.bmlp_last_error.restype = ctypes.c_char_p
            L.bmlp_default_options.argtypes = [ctypes.POINTER(bmlp_options)]
            L.bmlp_default_options.restype = None
            L.bmlp_get_stats.argtypes = [vp, ctypes.POINTER(bmlp_stats)]
            L.bmlp_rms.argtypes = [vp, vp, i64, i32, vp, ctypes.POINTER(bmlp_options), ctypes.POINTER(i32), vp]
            L.bmlp_rms_alg1.argtypes = [vp, vp, i64, i32, vp, ctypes.POINTER(bmlp_options), ctypes.POINTER(i32), vp]
            L.bmlp_smp.argtypes = [vp, vp, i64, i32, vp, i64, vp, ctypes.POINTER(bmlp_options),
                                   ctypes.POINTER(i32), vp]
            L.bmlp_compose.argtypes = [vp, vp, vp, i64, i32, vp, ctypes.POINTER(bmlp_options),
                                       ctypes.POINTER(i32), vp]
            L.bmlp_transpose.argtypes = [vp, vp, i64, i32, vp, vp]
            L.bmlp_union.argtypes = [vp, vp, vp, i64, i32, vp, vp]
            L.bmlp_negate.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
            L.bmlp_is_foreign.argtypes = [vp, vp, vp, vp, i64, i32, vp, ctypes.POINTER(bmlp_options),
                                          ctypes.POINTER(i32), vp]
            L.bmlp_mma_issue_rate.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_double)]
            L.bmlp_insert.argtypes = [vp, vp, i64, i32, vp, i64, vp]
            L.bmlp_batch_run.argtypes = [vp, ctypes.POINTER(bmlp_problem), i64, ctypes.POINTER(bmlp_options),
                                         ctypes.POINTER(i32), vp]
            L.bmlp_batch_autotune.argtypes = [vp, ctypes.POINTER(bmlp_problem), i64, ctypes.c_char_p, vp]
            fp, u8p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint8)
            L.bmlp_dispatch_features.argtypes = [vp, vp, i64, i32, fp, vp]
            L.bmlp_dispatch_train.argtypes = [vp, fp, fp, u8p, i64, ctypes.POINTER(bmlp_train_cfg), fp]
            L.bmlp_dispatch_predict.argtypes = [vp, fp, i64, fp, ctypes.POINTER(i32)]
            L.bmlp_dispatch_choose_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i32,
                                                    ctypes.POINTER(i32), fp, vp]
            L.bmlp_dispatch_loss_grad.argtypes = [vp, fp, fp, u8p, i64, fp, fp]
            L.bmlp_dispatch_set_params.argtypes = [vp, fp, fp, fp]
            L.bmlp_dispatch_get_params.argtypes = [vp, fp, fp, fp]
            L.bmlp_dispatch_save.argtypes = [vp, ctypes.c_char_p]
            L.bmlp_dispatch_load.argtypes = [vp, ctypes.c_char_p]
            for name in ("bmlp_ctx_create", "bmlp_ctx_destroy", "bmlp_get_stats", "bmlp_rms", "bmlp_smp",
                         "bmlp_compose", "bmlp_batch_run", "bmlp_batch_autotune", "bmlp_dispatch_features",
                         "bmlp_dispatch_train", "bmlp_dispatch_predict", "bmlp_dispatch_choose_many",
                         "bmlp_dispatch_loss_grad",
                         "bmlp_dispatch_set_params", "bmlp_dispatch_get_params", "bmlp_dispatch_save",
                         "bmlp_dispatch_load", "bmlp_transpose", "bmlp_union", "bmlp_negate", "bmlp_is_foreign",
                         "bmlp_mma_issue_rate", "bmlp_insert"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def header_functions():
    """Names of every function declared in include/bmlp.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bmlp_\w+)\s*\(", text)))


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):
        return ctypes.c_void_p(a.ctypes.data)
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError("expected a torch.Tensor, a numpy array or an int address")


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _u8ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _stream(stream, device):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_options(variant="auto", reflexive=False, max_iters=0, loop=BMLP_LOOP_HOST, profile=False, timeout_ns=0,
                 budget_ns=0, tc_only=False, e4m3_only=False):
    o = bmlp_options()
    lib().bmlp_default_options(ctypes.byref(o))
    o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    o.reflexive = int(bool(reflexive))
    o.max_iters = int(max_iters)
    o.loop = int(loop)
    o.profile = int(bool(profile))
    o.timeout_ns = int(timeout_ns)
    o.budget_ns = int(budget_ns)
    o.tc_only = int(bool(tc_only))
    o.e4m3_only = int(bool(e4m3_only))
    return o


class Context:
    """Owner of one ``bmlp_ctx`` on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self._L = lib()
        h = ctypes.c_void_p()
        st = self._L.bmlp_ctx_create(ctypes.byref(h), self.device)
        if st != BMLP_OK:
            raise BmlpError(st, "bmlp_ctx_create(device=%d) failed" % self.device)
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._L.bmlp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self) -> str:
        return self._L.bmlp_last_error(self.handle).decode()

    def _check(self, st):
        if st != BMLP_OK:
            raise BmlpError(st, self.last_error())

    def stats(self) -> dict:
        s = bmlp_stats()
        self._check(self._L.bmlp_get_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def rms(self, R, n, out, fmt=BMLP_FMT_U8, stream=None, **opt):
        """bmlp_rms: out = R1+ (or I + R1+). Returns the number of products."""
        o = make_options(**opt)
        it = ctypes.c_int32(0)
        self._check(self._L.bmlp_rms(self.handle, _ptr(R), int(n), int(fmt), _ptr(out), ctypes.byref(o),
                                     ctypes.byref(it), _stream(stream, self.device)))
        return it.value

    def rms_alg1(self, R, n, out, fmt=BMLP_FMT_U8, stream=None, **opt):
        """bmlp_rms_alg1: out = (I + R1)^(2^k) R1 = R1+ (Algorithm 1 as printed).
        Returns the squarings plus the final product."""
        o = make_options(**opt)
        it = ctypes.c_int32(0)
        self._check(self._L.bmlp_rms_alg1(self.handle, _ptr(R), int(n), int(fmt), _ptr(out), ctypes.byref(o),
                                          ctypes.byref(it), _stream(stream, self.device)))
        return it.value

    def smp(self, R, n, src_rows, q, out_rows, fmt=BMLP_FMT_U8, stream=None, **opt):
        """bmlp_smp: out_q = v_q R1+ for packed source rows. Returns the levels."""
        o = make_options(**opt)
        it = ctypes.c_int32(0)
        self._check(self._L.bmlp_smp(self.handle, _ptr(R), int(n), int(fmt), _ptr(src_rows), int(q), _ptr(out_rows),
                                     ctypes.byref(o), ctypes.byref(it), _stream(stream, self.device)))
        return it.value

    @staticmethod
    def problems(items):
        """ctypes array of bmlp_problem from dicts {kind, n, R1, R2, out, fmt, reflexive}."""
        arr = (bmlp_problem * max(len(items), 1))()
        for i, it in enumerate(items):
            p = arr[i]
            p.kind = int(it.get("kind", BMLP_PROBLEM_CLOSURE))
            p.fmt = int(it.get("fmt", BMLP_FMT_U8))
            p.reflexive = int(bool(it.get("reflexive", False)))
            v = it.get("variant", 0)
            p.variant = VARIANTS[v] if isinstance(v, str) else int(v)
            p.n = int(it["n"])
            p.R1 = _ptr(it["R1"]).value if it.get("R1") is not None else None
            p.R2 = _ptr(it["R2"]).value if it.get("R2") is not None else None
            p.out = _ptr(it["out"]).value if it.get("out") is not None else None
        return arr

    def batch_run(self, items, stream=None, **opt):
        """bmlp_batch_run over dicts (see ``problems``). Returns per-problem products."""
        arr = items if isinstance(items, ctypes.Array) else self.problems(items)
        count = len(items)
        o = make_options(**opt)
        iters = (ctypes.c_int32 * max(count, 1))()
        self._check(self._L.bmlp_batch_run(self.handle, arr, count, ctypes.byref(o), iters,
                                           _stream(stream, self.device)))
        return list(iters)[:count]

    def batch_autotune(self, items, cache_path=None, stream=None):
        """bmlp_batch_autotune: choose tensor cores or packed rows per size bucket."""
        arr = items if isinstance(items, ctypes.Array) else self.problems(items)
        path = cache_path.encode() if cache_path else None
        self._check(self._L.bmlp_batch_autotune(self.handle, arr, len(items), path, _stream(stream, self.device)))

    # ---------------------------------------------------- dispatcher --
    def dispatch_features(self, R, n, fmt=BMLP_FMT_U8, stream=None):
        """bmlp_dispatch_features: the 16 features (numpy float32)."""
        import numpy as np
        f = np.zeros(BMLP_NFEAT, np.float32)
        self._check(self._L.bmlp_dispatch_features(self.handle, _ptr(R), int(n), int(fmt), _fptr(f),
                                                   _stream(stream, self.device)))
        return f

    def dispatch_choose_many(self, mats, ns, fmt=BMLP_FMT_U8, stream=None, features=False):
        """bmlp_dispatch_choose_many: the chosen bmlp_variant of each matrix (numpy int32, m), and with
        features=True also their features (m x 16 float32); one host wait for all of them."""
        import numpy as np
        m = len(mats)
        ptrs = (ctypes.c_void_p * max(m, 1))(*[_ptr(a).value for a in mats])
        nn = (ctypes.c_int64 * max(m, 1))(*[int(x) for x in ns])
        choice = np.zeros(max(m, 1), np.int32)
        f = np.zeros((max(m, 1), BMLP_NFEAT), np.float32) if features else None
        self._check(self._L.bmlp_dispatch_choose_many(self.handle, ptrs, nn, m, int(fmt),
                                                      choice.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                      _fptr(f) if features else None,
                                                      _stream(stream, self.device)))
        return (choice[:m], f[:m]) if features else choice[:m]

    def dispatch_train(self, feats, log2_ms, censored, epochs=200, batch=256, lr=1e-3, weight_decay=1e-4, seed=0):
        """bmlp_dispatch_train on host arrays; returns the last epoch's loss."""
        import numpy as np
        X = np.ascontiguousarray(feats, np.float32)
        Y = np.ascontiguousarray(log2_ms, np.float32)
        C = np.ascontiguousarray(censored, np.uint8)
        cfg = bmlp_train_cfg(int(epochs), int(batch), float(lr), float(weight_decay), int(seed))
        loss = ctypes.c_float(0)
        self._check(self._L.bmlp_dispatch_train(self.handle, _fptr(X), _fptr(Y), _u8ptr(C), X.shape[0],
                                                ctypes.byref(cfg), ctypes.byref(loss)))
        return loss.value

    def dispatch_predict(self, feats):
        """bmlp_dispatch_predict: (pred m x 4 log2 ms, chosen bmlp_variant m)."""
        import numpy as np
        X = np.ascontiguousarray(np.atleast_2d(feats), np.float32)
        m = X.shape[0]
        pred = np.zeros((m, BMLP_NVAR), np.float32)
        choice = np.zeros(m, np.int32)
        self._check(self._L.bmlp_dispatch_predict(self.handle, _fptr(X), m, _fptr(pred),
                                                  choice.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return pred, choice

    def dispatch_loss_grad(self, feats, log2_ms, censored):
        import numpy as np
        X = np.ascontiguousarray(feats, np.float32)
        Y = np.ascontiguousarray(log2_ms, np.float32)
        C = np.ascontiguousarray(censored, np.uint8)
        g = np.zeros(BMLP_MLP_PARAMS, np.float32)
        loss = ctypes.c_float(0)
        self._check(self._L.bmlp_dispatch_loss_grad(self.handle, _fptr(X), _fptr(Y), _u8ptr(C), X.shape[0],
                                                    ctypes.byref(loss), _fptr(g)))
        return loss.value, g

    def dispatch_set_params(self, params=None, mu=None, sigma=None):
        import numpy as np
        a = [None if x is None else np.ascontiguousarray(x, np.float32) for x in (params, mu, sigma)]
        self._check(self._L.bmlp_dispatch_set_params(self.handle, *[_fptr(x) if x is not None else None for x in a]))

    def dispatch_get_params(self):
        import numpy as np
        p = np.zeros(BMLP_MLP_PARAMS, np.float32)
        mu = np.zeros(BMLP_NFEAT, np.float32)
        sg = np.zeros(BMLP_NFEAT, np.float32)
        self._check(self._L.bmlp_dispatch_get_params(self.handle, _fptr(p), _fptr(mu), _fptr(sg)))
        return p, mu, sg

    def dispatch_save(self, path):
        self._check(self._L.bmlp_dispatch_save(self.handle, str(path).encode()))

    def dispatch_load(self, path):
        self._check(self._L.bmlp_dispatch_load(self.handle, str(path).encode()))

    def compose(self, R1, R2, n, out, fmt=BMLP_FMT_U8, stream=None, **opt):
        """bmlp_compose: out = (I + R2+) R1. Returns the closure's products."""
        o = make_options(**opt)
        it = ctypes.c_int32(0)
        self._check(self._L.bmlp_compose(self.handle, _ptr(R1), _ptr(R2), int(n), int(fmt), _ptr(out),
                                         ctypes.byref(o), ctypes.byref(it), _stream(stream, self.device)))
        return it.value

    def transpose(self, R, n, out, fmt=BMLP_FMT_U8, stream=None):
        """bmlp_transpose (TRANSP): out = R^T."""
        self._check(self._L.bmlp_transpose(self.handle, _ptr(R), int(n), int(fmt), _ptr(out),
                                           _stream(stream, self.device)))

    def union(self, A, B, n, out, fmt=BMLP_FMT_U8, stream=None):
        """bmlp_union: out = A OR B."""
        self._check(self._L.bmlp_union(self.handle, _ptr(A), _ptr(B), int(n), int(fmt), _ptr(out),
                                       _stream(stream, self.device)))

    def negate(self, R, n, out, rows=None, cols=None, fmt=BMLP_FMT_U8, stream=None):
        """bmlp_negate (NEG): out = rows x cols AND NOT R (None = every constant)."""
        self._check(self._L.bmlp_negate(self.handle, _ptr(R), int(n), int(fmt), _ptr(rows), _ptr(cols), _ptr(out),
                                        _stream(stream, self.device)))

    def insert(self, closure, n, pairs, m=None, fmt=BMLP_FMT_U8, stream=None):
        """bmlp_insert: closure := (closure + pairs)+ in place; pairs is m x 2 int32."""
        if m is None:
            m = len(pairs)
        self._check(self._L.bmlp_insert(self.handle, _ptr(closure), int(n), int(fmt), _ptr(pairs), int(m),
                                        _stream(stream, self.device)))

    def mma_issue_rate(self, kind, iters=20000):
        """bmlp_mma_issue_rate: TFLOP/s of back-to-back tcgen05.mma (kind 0: E4M3 M128 N256 K32, 1: E2M1
        M128 N256 K64, 2: E2M1 M256 N256 K64 over a CTA pair, 4: E2M1 M256 N256 K64 + M256 N224 K64 over a CTA
        pair), or (kind 3) tera 64-bit word ORs per second."""
        v = ctypes.c_double(0.0)
        self._check(self._L.bmlp_mma_issue_rate(self.handle, int(kind), int(iters), ctypes.byref(v)))
        return v.value

    def is_foreign(self, contains, adjoins, n, out, location=None, fmt=BMLP_FMT_U8, stream=None, **opt):
        """bmlp_is_foreign: the composed program P3 u P4 u P5. Returns the
        products of (closure of contains, closure inside the composition)."""
        o = make_options(**opt)
        it = (ctypes.c_int32 * 2)()
        self._check(self._L.bmlp_is_foreign(self.handle, _ptr(contains), _ptr(adjoins), _ptr(location), int(n),
                                            int(fmt), _ptr(out), ctypes.byref(o), it, _stream(stream, self.device)))
        return it[0], it[1]


def rms_tc_noalloc(R, n, out, fmt=BMLP_FMT_U8, reflexive=False, max_iters=0, stream=None, device=0):
    """bmlp_rms_tc_noalloc: the tensor-core closure with no device allocation.

    For callers that must not allocate device memory (memory owned by a pool
    allocator or a fixed budget; latency-critical paths that cannot afford the
    device synchronisation of cudaMalloc / cudaFree). R and out must be device
    memory, n <= 2048. Returns the number of products; raises BmlpError.
    """
    L = lib()
    fn = L.bmlp_rms_tc_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    it = ctypes.c_int32(0)
    st = fn(_ptr(R), int(n), int(fmt), _ptr(out), int(bool(reflexive)), int(max_iters), ctypes.byref(it),
            _stream(stream, device))
    if st != BMLP_OK:
        raise BmlpError(st, "bmlp_rms_tc_noalloc failed")
    return it.value
