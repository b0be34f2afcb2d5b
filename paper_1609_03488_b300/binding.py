"""Thin ctypes binding of the C ABI declared in ``include/cvxb300.h``.

Argument marshalling only: every step of the SCS iteration runs in the CUDA
kernels of ``libcvxb300.so``.  Functions keep the C names; array arguments may
be NumPy arrays (host memory) or CUDA tensors (device memory, passed by
``data_ptr()``).  There is no fallback: if the shared library is missing this
module raises on import.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.lib_path()
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcvxb300.so not built ({LIB_PATH}); run python -m paper_1609_03488_b300.build")
lib = C.CDLL(LIB_PATH)

# ----------------------------------------------------------------- C types
CF_OK, CF_E_INVALID, CF_E_OOM, CF_E_CUDA, CF_E_BUSY, CF_E_TIMEOUT, CF_E_STATE = 0, -1, -2, -3, -4, -5, -6
CF_SOLVED, CF_INFEASIBLE, CF_UNBOUNDED, CF_MAX_ITERS, CF_NUMERICAL, CF_CANCELLED = range(6)
STATUS_NAMES = {0: "solved", 1: "infeasible", 2: "unbounded", 3: "max_iters", 4: "numerical", 5: "cancelled"}
CF_FP32, CF_BF16, CF_FP8_E4M3 = 0, 1, 2
PREC = {"fp32": CF_FP32, "bf16": CF_BF16, "fp8": CF_FP8_E4M3}
CF_VSTACK, CF_HSTACK, CF_BLOCKDIAG, CF_PRODUCT, CF_SUM, CF_SCALE, CF_ADJOINT, CF_KRON = range(8)
COMPOSE = {"vstack": CF_VSTACK, "hstack": CF_HSTACK, "blockdiag": CF_BLOCKDIAG,
           "product": CF_PRODUCT, "sum": CF_SUM, "scale": CF_SCALE, "adjoint": CF_ADJOINT,
           "kron": CF_KRON}


class cf_cone(C.Structure):
    _fields_ = [("z", C.c_int64), ("l", C.c_int64), ("q", C.POINTER(C.c_int64)), ("nq", C.c_int64)]


class cf_settings(C.Structure):
    _fields_ = [("eps", C.c_double), ("eps_infeas", C.c_double), ("alpha", C.c_double),
                ("max_iters", C.c_int32), ("check_interval", C.c_int32),
                ("cg_max_iters", C.c_int32), ("cg_fixed_iters", C.c_int32),
                ("cg_tol_rel", C.c_double), ("cg_tol_exp", C.c_double), ("cg_tol_min", C.c_double),
                ("setup_cg_max_iters", C.c_int32), ("setup_cg_tol", C.c_double),
                ("host_loop", C.c_int32), ("engine", C.c_int32)]


CF_ENGINE_AUTO, CF_ENGINE_GRAPH, CF_ENGINE_TEAM, CF_ENGINE_GRID = 0, 1, 2, 3
ENGINE = {"auto": CF_ENGINE_AUTO, "graph": CF_ENGINE_GRAPH, "team": CF_ENGINE_TEAM, "grid": CF_ENGINE_GRID}


class cf_schedule(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("threads", C.c_int32), ("csr_nnz_per_lane", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("team_bytes", C.c_double), ("auto_max_bytes", C.c_double),
                ("batch_max_bytes", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cf_tune_info(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("problems", C.c_int32), ("seconds", C.c_double),
                ("default_ms", C.c_double), ("best_ms", C.c_double), ("best", cf_schedule)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "best"}
        d["best"] = self.best.as_dict()
        return d


class cf_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("cg_iters_total", C.c_int64),
                ("checks", C.c_int32), ("setup_cg_iters", C.c_int32),
                ("pri_res", C.c_double), ("dual_res", C.c_double), ("gap", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("tau", C.c_double),
                ("kappa", C.c_double), ("setup_ns", C.c_int64), ("solve_ns", C.c_int64),
                ("kernel_launches", C.c_int64), ("queue_ns", C.c_int64), ("device_ns", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


P = C.c_void_p
PP = C.POINTER(C.c_void_p)
_sig = {
    "cf_settings_default": (None, [C.POINTER(cf_settings)]),
    "cf_ctx_create": (C.c_int, [C.c_int, P, PP]),
    "cf_ctx_destroy": (None, [P]),
    "cf_ctx_sm_count": (C.c_int, [P]),
    "cf_op_dense": (C.c_int, [P, C.c_int64, C.c_int64, P, C.c_int, PP]),
    "cf_op_csr": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64, P, P, P, C.c_int, PP]),
    "cf_op_conv1d": (C.c_int, [P, C.c_int64, P, C.c_int64, PP]),
    "cf_op_conv1d_method": (C.c_int, [P, C.c_int64, P, C.c_int64, C.c_int32, PP]),
    "cf_op_conv2d": (C.c_int, [P, C.c_int64, C.c_int64, P, C.c_int64, C.c_int64, PP]),
    "cf_op_diag": (C.c_int, [P, C.c_int64, P, PP]),
    "cf_op_zero": (C.c_int, [P, C.c_int64, C.c_int64, PP]),
    "operator_compose": (C.c_int, [P, C.c_int, PP, C.c_int32, C.c_double, PP]),
    "cf_op_kron": (C.c_int, [P, P, P, PP]),
    "cf_op_destroy": (None, [P]),
    "cf_op_shape": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "cf_op_apply": (C.c_int, [P, C.c_int32, P, P]),
    "cf_op_dense_stored": (C.c_int, [P, P, P]),
    "cf_op_apply_async": (C.c_int, [P, C.c_int32, C.c_float, P, P, C.c_int32, P, P]),
    "cf_op_workspace_bytes": (C.c_int, [P, C.c_int32, C.POINTER(C.c_size_t)]),
    "cf_op_apply_static": (C.c_int, [P, C.c_int32, C.c_float, P, P, C.c_int32, P]),
    "cone_problem_create": (C.c_int, [P, P, P, C.c_int64, P, C.c_int64, C.POINTER(cf_cone), PP]),
    "cf_problem_destroy": (None, [P]),
    "solve": (C.c_int, [P, C.POINTER(cf_settings), P, P, P, P, P, C.POINTER(cf_info)]),
    "solve_batch": (C.c_int, [PP, C.c_int32, C.POINTER(cf_settings), PP, PP, PP, C.POINTER(cf_info)]),
    "solve_batch_tune": (C.c_int, [PP, C.c_int32, C.c_int32, C.POINTER(cf_tune_info)]),
    "cf_ctx_get_schedule": (C.c_int, [P, C.POINTER(cf_schedule)]),
    "cf_ctx_set_schedule": (C.c_int, [P, C.POINTER(cf_schedule)]),
    "cf_problem_team_info": (C.c_int, [P, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_char_p,
                                       C.c_size_t]),
    "cone_problem_equilibrate": (C.c_int, [P, C.c_int32, C.c_int32, C.c_uint64]),
    "cone_problem_set_inner": (C.c_int, [P, P]),
    "cf_problem_scaling": (C.c_int, [P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "cg_solve": (C.c_int, [P, C.c_double, P, P, C.c_int32, C.c_double, C.POINTER(C.c_int32),
                           C.POINTER(C.c_double)]),
    "serve_create": (C.c_int, [P, C.c_size_t, C.c_int32, PP]),
    "serve_submit": (C.c_int, [P, P, C.POINTER(cf_settings), C.POINTER(C.c_int64)]),
    "serve_wait": (C.c_int, [P, C.c_int64, C.c_int64, P, P, P, C.POINTER(cf_info)]),
    "serve_destroy": (None, [P]),
    "cf_measure_fma_rate": (C.c_int, [P, C.c_int32, C.POINTER(C.c_double)]),
    "cf_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_sig)


class CfError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.cf_last_error().decode(errors="replace")
        super().__init__(f"{where}: error {code}: {msg}")
        self.code = code


def check(code, where):
    if code != CF_OK:
        raise CfError(code, where)
    return code


def cf_last_error():
    return lib.cf_last_error().decode(errors="replace")


# ------------------------------------------------------------ marshalling
def _ptr(a):
    """Address of a NumPy array or a CUDA tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _f32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def cf_settings_default():
    s = cf_settings()
    lib.cf_settings_default(C.byref(s))
    return s


def settings(**kw):
    s = cf_settings_default()
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        if k == "engine" and isinstance(v, str):
            v = ENGINE[v]
        setattr(s, k, v)
    return s


def get_schedule(ctx):
    s = cf_schedule()
    check(lib.cf_ctx_get_schedule(ctx.h, C.byref(s)), "cf_ctx_get_schedule")
    return s.as_dict()


def set_schedule(ctx, **kw):
    """Change fields of the context's team-engine schedule."""
    s = cf_schedule()
    check(lib.cf_ctx_get_schedule(ctx.h, C.byref(s)), "cf_ctx_get_schedule")
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    check(lib.cf_ctx_set_schedule(ctx.h, C.byref(s)), "cf_ctx_set_schedule")
    return s.as_dict()


class Context:
    """cf_ctx_create(device, stream).  ``stream`` is a cudaStream_t handle
    (int) or None for a context-owned stream."""

    def __init__(self, device=0, stream=None):
        h = C.c_void_p()
        check(lib.cf_ctx_create(device, C.c_void_p(stream) if stream else None, C.byref(h)), "cf_ctx_create")
        self.h = h
        self.device = device

    @property
    def sm_count(self):
        return lib.cf_ctx_sm_count(self.h)

    def fma_rate(self, fp64=False):
        """cf_measure_fma_rate: measured FMA rate of the GPU in flop/s."""
        v = C.c_double()
        check(lib.cf_measure_fma_rate(self.h, 1 if fp64 else 0, C.byref(v)), "cf_measure_fma_rate")
        return v.value

    def close(self):
        if self.h:
            lib.cf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """Owning handle of a cf_op."""

    def __init__(self, ctx, h, keep=()):
        self.ctx, self.h, self._keep = ctx, h, keep
        m, n = C.c_int64(), C.c_int64()
        check(lib.cf_op_shape(h, C.byref(m), C.byref(n)), "cf_op_shape")
        self.m, self.n = m.value, n.value

    def apply(self, x, adjoint=False, out=None):
        """cf_op_apply: y = A x or A^T x (float32, host or device)."""
        x = _f32(x)
        if out is None:
            out = np.empty(self.n if adjoint else self.m, dtype=np.float32)
        check(lib.cf_op_apply(self.h, 1 if adjoint else 0, _ptr(x), _ptr(out)), "cf_op_apply")
        return out

    def workspace_bytes(self, adjoint=False):
        b = C.c_size_t()
        check(lib.cf_op_workspace_bytes(self.h, 1 if adjoint else 0, C.byref(b)), "cf_op_workspace_bytes")
        return b.value

    def apply_async(self, x, y, adjoint=False, alpha=1.0, accumulate=False, workspace=None, stream=None):
        """cf_op_apply_async on device tensors; returns immediately."""
        check(lib.cf_op_apply_async(self.h, 1 if adjoint else 0, float(alpha), _ptr(x), _ptr(y),
                                    1 if accumulate else 0, _ptr(workspace),
                                    C.c_void_p(stream) if stream else None), "cf_op_apply_async")

    def apply_static(self, x, y, adjoint=False, alpha=1.0, accumulate=False, stream=None):
        """cf_op_apply_static on device tensors (scratch from the library's
        static device array; nothing is allocated).  Without ``stream`` the
        call is enqueued on torch's current stream of x's device, so it is
        ordered after the torch kernels that produced x and y."""
        if stream is None and hasattr(x, "device"):
            import torch
            stream = torch.cuda.current_stream(x.device).cuda_stream
        check(lib.cf_op_apply_static(self.h, 1 if adjoint else 0, float(alpha), _ptr(x), _ptr(y),
                                     1 if accumulate else 0, C.c_void_p(stream) if stream else None),
              "cf_op_apply_static")

    def dense_stored(self, prec):
        """cf_op_dense_stored: the stored codes (and FP8 row scales)."""
        dt = {CF_FP32: np.float32, CF_BF16: np.uint16, CF_FP8_E4M3: np.uint8}[prec]
        codes = np.empty((self.m, self.n), dtype=dt)
        scales = np.empty(self.m, dtype=np.float32) if prec == CF_FP8_E4M3 else None
        check(lib.cf_op_dense_stored(self.h, _ptr(codes), _ptr(scales)), "cf_op_dense_stored")
        return codes, scales

    def close(self):
        if self.h:
            lib.cf_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _new(fn, *args):
    h = C.c_void_p()
    check(getattr(lib, fn)(*args, C.byref(h)), fn)
    return h


def cf_op_dense(ctx, data, storage="fp32"):
    data = _f32(data)
    m, n = data.shape
    return Operator(ctx, _new("cf_op_dense", ctx.h, m, n, _ptr(data), PREC[storage]))


def cf_op_csr(ctx, m, n, rowptr, col, val, storage="fp32"):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f32(val)
    return Operator(ctx, _new("cf_op_csr", ctx.h, m, n, len(col), _ptr(rowptr), _ptr(col), _ptr(val),
                              PREC[storage]))


CONV_METHOD = {"auto": 0, "direct": 1, "fft": 2}


def cf_op_conv1d(ctx, kernel, n, method="auto"):
    """1-D full convolution leaf; method "auto", "direct" or "fft"
    (cf_op_conv1d_method)."""
    kernel = _f32(kernel)
    return Operator(ctx, _new("cf_op_conv1d_method", ctx.h, n, _ptr(kernel), kernel.size, CONV_METHOD[method]))


def cf_op_conv2d(ctx, kernel, h, w):
    kernel = _f32(kernel)
    kh, kw = kernel.shape
    return Operator(ctx, _new("cf_op_conv2d", ctx.h, h, w, _ptr(kernel), kh, kw))


def cf_op_diag(ctx, n, d=None):
    return Operator(ctx, _new("cf_op_diag", ctx.h, n, _ptr(_f32(d))))


def cf_op_zero(ctx, m, n):
    return Operator(ctx, _new("cf_op_zero", ctx.h, m, n))


def operator_compose(ctx, kind, parts, alpha=1.0):
    arr = (C.c_void_p * len(parts))(*[p.h.value for p in parts])
    h = _new("operator_compose", ctx.h, COMPOSE[kind], arr, len(parts), float(alpha))
    return Operator(ctx, h)


def cf_op_kron(ctx, A, Bop):
    """cf_op_kron: A (x) B of two dense FP32 operators."""
    return Operator(ctx, _new("cf_op_kron", ctx.h, A.h, Bop.h), keep=(A, Bop))


def build_operator(ctx, node):
    """Create the cf_op tree for an operator-tree description (the format of
    the synthetic input generator): one C call per node."""
    k = node["kind"]
    if k == "dense":
        return cf_op_dense(ctx, node["data"], node["storage"])
    if k == "csr":
        return cf_op_csr(ctx, node["m"], node["n"], node["rowptr"], node["col"], node["val"],
                         node.get("storage", "fp32"))
    if k == "conv1d":
        return cf_op_conv1d(ctx, node["kernel"], node["n"], node.get("method", "auto"))
    if k == "conv2d":
        return cf_op_conv2d(ctx, node["kernel"], node["h"], node["w"])
    if k == "diag":
        return cf_op_diag(ctx, node["n"], node["d"])
    if k == "zero":
        return cf_op_zero(ctx, node["m"], node["n"])
    parts = [build_operator(ctx, p) for p in node["parts"]]
    return operator_compose(ctx, k, parts, node.get("alpha", 1.0))


class Problem:
    """cone_problem_create over an Operator; keeps the operator alive."""

    def __init__(self, ctx, op, b, c, cone):
        self.ctx, self.op = ctx, op
        b, c = _f64(b), _f64(c)
        q = np.ascontiguousarray(cone.get("q", []), dtype=np.int64)
        self._q = q
        cc = cf_cone(int(cone.get("z", 0)), int(cone.get("l", 0)),
                     q.ctypes.data_as(C.POINTER(C.c_int64)) if q.size else None, q.size)
        self.m, self.n = op.m, op.n
        self.h = _new("cone_problem_create", ctx.h, op.h, _ptr(b), self.m, _ptr(c), self.n, C.byref(cc))

    def close(self):
        if self.h:
            lib.cf_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cone_problem_create(ctx, prob):
    """Problem from a generator problem dict (builds its operator tree)."""
    return Problem(ctx, build_operator(ctx, prob["A"]), prob["b"], prob["c"], prob["cone"])


def solve(problem, st=None, x=None, y=None, s=None, warm_uv=None, uv_out=None):
    """solve(): returns (info dict, x, y, s[, uv]) with NumPy outputs unless
    caller buffers are given."""
    n, m = problem.n, problem.m
    if x is None:
        x = np.empty(n)
    if y is None:
        y = np.empty(m)
    if s is None:
        s = np.empty(m)
    info = cf_info()
    check(lib.solve(problem.h, C.byref(st) if st is not None else None, _ptr(x), _ptr(y), _ptr(s),
                    _ptr(_f64(warm_uv)), _ptr(uv_out), C.byref(info)), "solve")
    return info.as_dict(), x, y, s


def solve_batch(problems, st=None):
    k = len(problems)
    hs = (C.c_void_p * k)(*[p.h.value for p in problems])
    xs = [np.empty(p.n) for p in problems]
    ys = [np.empty(p.m) for p in problems]
    ss = [np.empty(p.m) for p in problems]
    px = (C.c_void_p * k)(*[a.ctypes.data for a in xs])
    py = (C.c_void_p * k)(*[a.ctypes.data for a in ys])
    ps = (C.c_void_p * k)(*[a.ctypes.data for a in ss])
    infos = (cf_info * k)()
    check(lib.solve_batch(hs, k, C.byref(st) if st is not None else None, px, py, ps, infos), "solve_batch")
    return [i.as_dict() for i in infos], xs, ys, ss


def equilibrate(problem, iters=10, probes=8, seed=0x5EED):
    """cone_problem_equilibrate: scale the problem's data (see the header)."""
    check(lib.cone_problem_equilibrate(problem.h, int(iters), int(probes), int(seed)), "cone_problem_equilibrate")


def set_inner(problem, inner):
    """cone_problem_set_inner: ``inner`` is an Operator, an operator tree
    (built here, e.g. ``synth.with_storage(prob["A"], "fp8")``) or None."""
    if isinstance(inner, dict):
        inner = build_operator(problem.ctx, inner)
    check(lib.cone_problem_set_inner(problem.h, inner.h if inner is not None else None), "cone_problem_set_inner")
    return inner


def scaling(problem):
    """(D, E, sigma, rho) of a problem's equilibration."""
    D = np.empty(problem.m, dtype=np.float32)
    E = np.empty(problem.n, dtype=np.float32)
    sg, rh = C.c_double(), C.c_double()
    check(lib.cf_problem_scaling(problem.h, _ptr(D), _ptr(E), C.byref(sg), C.byref(rh)), "cf_problem_scaling")
    return D, E, sg.value, rh.value


def team_info(problem):
    """(supported, pass_bytes, why) of the team engine for a problem."""
    ok, nb = C.c_int32(), C.c_double()
    buf = C.create_string_buffer(256)
    check(lib.cf_problem_team_info(problem.h, C.byref(ok), C.byref(nb), buf, 256), "cf_problem_team_info")
    return bool(ok.value), nb.value, buf.value.decode()


def solve_batch_tune(problems, iters=20):
    k = len(problems)
    hs = (C.c_void_p * k)(*[p.h.value for p in problems])
    info = cf_tune_info()
    check(lib.solve_batch_tune(hs, k, int(iters), C.byref(info)), "solve_batch_tune")
    return info.as_dict()


def cg_solve(op, lam, rhs, x0=None, max_iters=1000, tol=1e-8):
    rhs = _f32(rhs)
    x = np.zeros(op.n, dtype=np.float32) if x0 is None else _f32(np.array(x0, copy=True))
    it = C.c_int32()
    rn = C.c_double()
    check(lib.cg_solve(op.h, float(lam), _ptr(rhs), _ptr(x), int(max_iters), float(tol), C.byref(it),
                       C.byref(rn)), "cg_solve")
    return x, it.value, rn.value


class Server:
    def __init__(self, ctx, budget_bytes, max_slots):
        self.ctx = ctx
        self.h = _new("serve_create", ctx.h, int(budget_bytes), int(max_slots))

    def submit(self, problem, st=None):
        t = C.c_int64()
        check(lib.serve_submit(self.h, problem.h, C.byref(st) if st is not None else None, C.byref(t)),
              "serve_submit")
        return t.value

    def wait(self, ticket, problem, timeout_ns=-1):
        x, y, s = np.empty(problem.n), np.empty(problem.m), np.empty(problem.m)
        info = cf_info()
        check(lib.serve_wait(self.h, ticket, timeout_ns, _ptr(x), _ptr(y), _ptr(s), C.byref(info)),
              "serve_wait")
        return info.as_dict(), x, y, s

    def close(self):
        if self.h:
            lib.serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
