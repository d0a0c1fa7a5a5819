"""ctypes binding of libils.so: argument marshalling only.

The functions keep the C names of ``include/ils.h``.  Device pointers, leading
dimensions and the stream are passed as plain integers; the small ``Solver``
wrapper takes torch CUDA tensors and reads their pointers.  Every numerical step
runs inside the CUDA library; if ``libils.so`` is missing this module raises
instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libils.so")

ILS_OK = 0
ILS_ERR_INVALID_ARG = 1
ILS_ERR_NOT_SPD = 2
ILS_ERR_NO_CONVERGENCE = 3
ILS_ERR_NONFINITE = 4
ILS_ERR_TIMEOUT = 5
ILS_ERR_CUDA = 6
ILS_ERR_OOM = 7

ILS_SP = 0
ILS_SP_RK_RGS = 1
ILS_SP_SCD = 2

ILS_FP64 = 0
ILS_FP32_REFINE = 1
ILS_BF16_REFINE = 2

ILS_ROUTE_AUTO = 0
ILS_ROUTE_EXPLICIT = 1
ILS_ROUTE_MATRIX_FREE = 2

ILS_GRAM_FP64 = 0
ILS_GRAM_SPLIT = 1

ILS_STOP_RELRES = 0
ILS_STOP_PAPER_RR = 1
ILS_STOP_ERR_BOUND = 2

MAT_GRAM1, MAT_GRAM2, MAT_CHOL, MAT_P, MAT_B = range(5)


class ils_options(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("gram", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("max_outer", ctypes.c_int64),
        ("max_inner", ctypes.c_int64),
        ("theta", ctypes.c_double),
        ("check_every", ctypes.c_int64),
        ("scd_sampler", ctypes.c_int32),
        ("sweeps", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("route", ctypes.c_int32),
        ("chain_ctas", ctypes.c_int32),
        ("stop_rule", ctypes.c_int32),
        ("estimate", ctypes.c_int32),
        ("alpha_mode", ctypes.c_int32),
        ("sampler", ctypes.c_int32),
        ("alpha_fixed", ctypes.c_int64),
        ("warm_inner", ctypes.c_int32),
        ("inner_form", ctypes.c_int32),
        ("tune_cache", ctypes.c_char_p),
        ("wait_limit_ns", ctypes.c_int64),
        ("lanczos_steps", ctypes.c_int32),
        ("factor64", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("theta_decay", ctypes.c_double),
        ("theta_min", ctypes.c_double),
    ]


class ils_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64), ("q", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64)]


class ils_info(ctypes.Structure):
    _fields_ = [
        ("outer_iters", ctypes.c_int64),
        ("inner_iters", ctypes.c_int64),
        ("refinements", ctypes.c_int64),
        ("relres", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("err_bound", ctypes.c_double),
        ("rho_est", ctypes.c_double),
        ("kappa_est", ctypes.c_double),
        ("t_setup_ms", ctypes.c_double),
        ("t_solve_ms", ctypes.c_double),
        ("t_inner_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if not f[0].startswith("reserved")}


# Exported symbols and their ctypes signatures, in the order of include/ils.h.
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
SIGNATURES = {
    "ils_options_default": (ctypes.c_int, [ctypes.POINTER(ils_options)]),
    "ils_setup": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64, _I64, _P, _I64,
                                 ctypes.POINTER(ils_options), _P]),
    "ils_setup_csr": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64, _I64, _I64, _P, _P, _P,
                                     ctypes.POINTER(ils_options), _P]),
    "ils_refactor": (ctypes.c_int, [_P, _P, _I64, _P]),
    "ils_refactor_async": (ctypes.c_int, [_P, _P, _I64, _P]),
    "ils_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ils_info), _P]),
    "ils_solve_many": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _I64, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(ils_info), _P]),
    "ils_get_matrix": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _P]),
    "ils_aq_product": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "ils_get_timings": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "ils_kernel_launches": (ctypes.c_int64, []),
    "ils_tuned_shape": (ctypes.c_int, [_I64, _I64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "ils_batch_setup": (ctypes.c_int, [ctypes.POINTER(_P), _I64, ctypes.POINTER(ils_problem),
                                       ctypes.POINTER(ils_options), _P]),
    "ils_batch_solve": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                       ctypes.POINTER(_I64), ctypes.c_int, ctypes.c_double, ctypes.POINTER(ils_info),
                                       _P]),
    "ils_batch_capture": (ctypes.c_int, [_P, ctypes.c_int, _I64, ctypes.POINTER(_P), ctypes.POINTER(_I64),
                                         ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.c_int, ctypes.c_double,
                                         _I64, _P]),
    "ils_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(ils_info), _P]),
    "ils_batch_handle": (_P, [_P, _I64]),
    "ils_batch_destroy": (None, [_P]),
    "ils_mlp_create": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64, ctypes.c_uint64, _P]),
    "ils_mlp_num_params": (_I64, [_P]),
    "ils_mlp_get_params": (ctypes.c_int, [_P, _P, _P]),
    "ils_mlp_set_params": (ctypes.c_int, [_P, _P, _P]),
    "ils_mlp_loss_grad": (ctypes.c_int, [_P, _I64, _P, _P, ctypes.POINTER(ctypes.c_double), _P, _P]),
    "ils_mlp_train": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _I64, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                     _P]),
    "ils_mlp_forward": (ctypes.c_int, [_P, _I64, _P, _P, _I64, ctypes.c_int, _P]),
    "ils_solve_param": (ctypes.c_int, [_P, _P, _I64, _P, _P, _I64, _P, _I64, ctypes.c_double,
                                       ctypes.POINTER(ils_info), _P]),
    "ils_mlp_destroy": (None, [_P]),
    "ils_set_warmstart": (ctypes.c_int, [_P, _P]),
    "ils_gram_noalloc": (ctypes.c_int, [_I64, _I64, _P, _I64, _P, _I64, _P]),
    "ils_route_model": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "ils_set_wait_limit": (ctypes.c_int, [_P, _I64]),
    "ils_record_picks": (ctypes.c_int, [_P, _P, _I64]),
    "ils_destroy": (None, [_P]),
    "ils_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ils_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libils.so (built by ``__graft_entry__.build()``); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first (python -c "
                "'import __graft_entry__ as g; g.build()'). There is no CPU fallback.")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def kernel_launches() -> int:
    """Kernels launched by libils.so in this process so far."""
    return int(lib().ils_kernel_launches())


def tuned_shape(n: int, k: int, bf16: bool = False):
    """(warps per CTA, CTAs) the autotuner picked for the sweep of an n x n operator, or None."""
    w, b = ctypes.c_int(), ctypes.c_int()
    if lib().ils_tuned_shape(n, k, int(bool(bf16)), ctypes.byref(w), ctypes.byref(b)):
        return w.value, b.value
    return None


def route_model():
    """The last automatic route decision: dict of modelled costs, measured rates and the choice."""
    buf = (ctypes.c_double * 9)()
    n = lib().ils_route_model(buf, 9)
    keys = ["explicit_s", "matrix_free_s", "gram_split_flops", "gram_f64_flops", "bw_fp64", "bw_fp32", "bw_bf16",
            "copy_Bps", "matrix_free"]
    return {k: buf[i] for i, k in enumerate(keys[:max(n, 0)])}


def status_string(code: int) -> str:
    return lib().ils_status_string(int(code)).decode()


class ILSError(RuntimeError):
    def __init__(self, code: int, where: str):
        detail = ""
        if code == ILS_ERR_CUDA:
            detail = " [" + lib().ils_last_error().decode(errors="replace") + "]"
        super().__init__(f"{where}: {status_string(code)} (status {code}){detail}")
        self.code = code


def _check(code: int, where: str, allow=(ILS_OK,)):
    if code not in allow:
        raise ILSError(code, where)
    return code


def options(**kw) -> ils_options:
    o = ils_options()
    _check(lib().ils_options_default(ctypes.byref(o)), "ils_options_default")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _colmajor_ptr(t, rows: int, cols: int) -> tuple:
    """Device pointer and leading dimension of a column-major rows x cols matrix.

    A torch tensor of shape (cols, rows) with unit stride along its last axis is
    the column-major layout the C ABI expects (it is the transpose view of a
    row-major tensor).
    """
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if t.dtype.itemsize != 8:
        raise ValueError("FP64 tensor expected")
    if t.dim() == 1:
        if t.shape[0] != rows or t.stride(0) != 1:
            raise ValueError("vector shape/stride mismatch")
        return t.data_ptr(), rows
    if tuple(t.shape) != (cols, rows) or t.stride(1) != 1:
        raise ValueError(f"expected a ({cols}, {rows}) tensor with unit inner stride, got "
                         f"{tuple(t.shape)} strides {t.stride()}")
    return t.data_ptr(), t.stride(0)


class Solver:
    """One ILS instance on the GPU (wraps an ils_handle).

    ``At`` holds A column-major: a CUDA float64 tensor of shape (n, m).
    """

    def __init__(self, At, p: int, opts: ils_options | None = None, stream=None):
        n, m = At.shape
        self.m, self.n, self.p, self.q = m, n, p, m - p
        ptr, lda = _colmajor_ptr(At, m, n)
        self.opts = opts if opts is not None else options()
        h = ctypes.c_void_p()
        code = lib().ils_setup(ctypes.byref(h), m, n, p, m - p, ptr, lda, ctypes.byref(self.opts),
                               _stream_ptr(stream))
        _check(code, "ils_setup")
        self.h = h

    @classmethod
    def from_csr(cls, m: int, n: int, p: int, rowptr, colind, val, opts: ils_options | None = None,
                 stream=None):
        """Instance with a sparse A given in CSR: CUDA tensors rowptr (int32, m + 1),
        colind (int32, nnz) and val (float64, nnz); rows 0..p-1 form A_1."""
        for t, dt in ((rowptr, 4), (colind, 4), (val, 8)):
            if not t.is_cuda or t.dtype.itemsize != dt or t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
                raise ValueError("rowptr/colind must be contiguous int32 and val contiguous float64 CUDA vectors")
        if rowptr.numel() != m + 1 or colind.numel() != val.numel():
            raise ValueError("CSR array lengths do not match")
        self = cls.__new__(cls)
        self.m, self.n, self.p, self.q = m, n, p, m - p
        self.opts = opts if opts is not None else options()
        h = ctypes.c_void_p()
        code = lib().ils_setup_csr(ctypes.byref(h), m, n, p, m - p, int(val.numel()), rowptr.data_ptr(),
                                   colind.data_ptr(), val.data_ptr(), ctypes.byref(self.opts), _stream_ptr(stream))
        _check(code, "ils_setup_csr")
        self.h = h
        return self

    def refactor(self, At, stream=None):
        ptr, lda = _colmajor_ptr(At, self.m, self.n)
        return _check(lib().ils_refactor(self.h, ptr, lda, _stream_ptr(stream)), "ils_refactor")

    def refactor_async(self, At, stream=None):
        """Enqueue the setup for new values of A; the next solve reports its status.

        That solve may form A^T J b before the setup ends, so its right-hand sides must be in
        place when this is called (not written by work enqueued between the two calls)."""
        ptr, lda = _colmajor_ptr(At, self.m, self.n)
        return _check(lib().ils_refactor_async(self.h, ptr, lda, _stream_ptr(stream)), "ils_refactor_async")

    def solve(self, b, x, x0_zero=True, tol=1e-12, stream=None, allow=(ILS_OK,)):
        """Solve into the CUDA tensor ``x`` (length n) for ``b`` (length m)."""
        bp, _ = _colmajor_ptr(b, self.m, 1)
        xp, _ = _colmajor_ptr(x, self.n, 1)
        info = ils_info()
        code = lib().ils_solve(self.h, bp, xp, int(bool(x0_zero)), float(tol), ctypes.byref(info),
                               _stream_ptr(stream))
        _check(code, "ils_solve", allow)
        return info

    def solve_many(self, Bt, Xt, x0_zero=True, tol=1e-12, stream=None, allow=(ILS_OK,)):
        """k right-hand sides: ``Bt`` (k, m) and ``Xt`` (k, n), both column-major views."""
        k = Bt.shape[0]
        bp, ldb = _colmajor_ptr(Bt, self.m, k)
        xp, ldx = _colmajor_ptr(Xt, self.n, k)
        info = ils_info()
        code = lib().ils_solve_many(self.h, k, bp, ldb, xp, ldx, int(bool(x0_zero)), float(tol),
                                    ctypes.byref(info), _stream_ptr(stream))
        _check(code, "ils_solve_many", allow)
        return info

    def aq_product(self, x, v, prec=0, stream=None):
        """v = A_2^T (A_2 x) by the one-pass stream (prec 0 the FP64-accurate copy: FP64, or
        double-FP32 on a mixed-precision handle; 1 the FP32 copy, 2 the BF16 copy)."""
        return _check(lib().ils_aq_product(self.h, x.data_ptr(), v.data_ptr(), prec, _stream_ptr(stream)),
                      "ils_aq_product")

    def record_picks(self, picks):
        """Record the first chain's picks of the first outer iteration into the int32 CUDA
        tensor `picks` (None stops recording); see ils_record_picks."""
        ptr = None if picks is None else picks.data_ptr()
        cap = 0 if picks is None else picks.numel()
        return _check(lib().ils_record_picks(self.h, ptr, cap), "ils_record_picks")

    def set_wait_limit(self, ns: int):
        """ils_set_wait_limit: bound (ns) on the one-launch solve's barrier waits; 0 = default."""
        return _check(lib().ils_set_wait_limit(self.h, int(ns)), "ils_set_wait_limit")

    def set_warmstart(self, net):
        """Attach a WarmStartNet (None detaches) for solve_param calls without a network."""
        return _check(lib().ils_set_warmstart(self.h, None if net is None else net.h), "ils_set_warmstart")

    def solve_param(self, theta, Bt, Xt, tol=1e-12, stream=None, allow=(ILS_OK,)):
        """ils_solve_param with the attached network (ils_set_warmstart)."""
        k = Bt.shape[0]
        bp, ldb = _colmajor_ptr(Bt, self.m, k)
        xp, ldx = _colmajor_ptr(Xt, self.n, k)
        info = ils_info()
        code = lib().ils_solve_param(self.h, None, k, theta.data_ptr(), bp, ldb, xp, ldx, float(tol),
                                     ctypes.byref(info), _stream_ptr(stream))
        _check(code, "ils_solve_param", allow)
        return info

    def get_matrix(self, which: int, out, stream=None):
        ptr, ld = _colmajor_ptr(out, self.n, self.n)
        return _check(lib().ils_get_matrix(self.h, which, ptr, ld, _stream_ptr(stream)), "ils_get_matrix")

    def timings(self):
        """Setup phase times (ms) of the last setup/refactor and of the last solve, when
        options.timing was set."""
        buf = (ctypes.c_double * 14)()
        n = lib().ils_get_timings(self.h, buf, 14)
        keys = ["gram1", "gram2", "factor", "products", "setup", "copy_A", "gram1_mma", "solve_start_gap",
                "solve_work", "solve_copy", "kappa_start", "kappa", "grams_done", "h_formed"]
        return {k: buf[i] for i, k in enumerate(keys[:max(n, 0)])}

    def close(self):
        if getattr(self, "h", None):
            lib().ils_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """A batch of independent ILS instances (wraps an ils_batch).

    ``Ats`` is a list of CUDA float64 tensors of shape (n_i, m_i) (A_i column-major) and
    ``ps`` the list of p_i.
    """

    def __init__(self, Ats, ps, opts: ils_options | None = None, stream=None):
        count = len(Ats)
        probs = (ils_problem * count)()
        self.shapes = []
        for i, (At, p) in enumerate(zip(Ats, ps)):
            n, m = At.shape
            ptr, lda = _colmajor_ptr(At, m, n)
            probs[i] = ils_problem(m, n, p, m - p, ptr, lda)
            self.shapes.append((m, n, p))
        self._keep = Ats
        self.opts = opts if opts is not None else options()
        b = ctypes.c_void_p()
        _check(lib().ils_batch_setup(ctypes.byref(b), count, probs, ctypes.byref(self.opts), _stream_ptr(stream)),
               "ils_batch_setup")
        self.b = b
        self.count = count

    def solve(self, Bts, Xts, x0_zero=True, tol=1e-12, stream=None, allow=(ILS_OK,)):
        """Bts[i]: (k, m_i) tensor, Xts[i]: (k, n_i) tensor, column-major views."""
        count = self.count
        k = Bts[0].shape[0]
        Bp = (ctypes.c_void_p * count)()
        Xp = (ctypes.c_void_p * count)()
        lb = (ctypes.c_int64 * count)()
        lx = (ctypes.c_int64 * count)()
        for i, ((m, n, _), Bt, Xt) in enumerate(zip(self.shapes, Bts, Xts)):
            Bp[i], lb[i] = _colmajor_ptr(Bt, m, k)
            Xp[i], lx[i] = _colmajor_ptr(Xt, n, k)
        infos = (ils_info * count)()
        code = lib().ils_batch_solve(self.b, k, Bp, lb, Xp, lx, int(bool(x0_zero)), float(tol), infos,
                                     _stream_ptr(stream))
        _check(code, "ils_batch_solve", allow)
        return list(infos)

    def _ptrs(self, Bts, Xts):
        count = self.count
        k = Bts[0].shape[0]
        Bp = (ctypes.c_void_p * count)()
        Xp = (ctypes.c_void_p * count)()
        lb = (ctypes.c_int64 * count)()
        lx = (ctypes.c_int64 * count)()
        for i, ((m, n, _), Bt, Xt) in enumerate(zip(self.shapes, Bts, Xts)):
            Bp[i], lb[i] = _colmajor_ptr(Bt, m, k)
            Xp[i], lx[i] = _colmajor_ptr(Xt, n, k)
        return k, Bp, lb, Xp, lx

    def capture(self, Bts, Xts, refactor=False, steps=8, x0_zero=True, tol=1e-12, stream=None):
        """Record the batch solve (and, with refactor, the setup) as one CUDA graph.  The
        tensors must stay alive: the graph reads and writes them at their addresses.
        ``stream`` must be a non-default torch stream."""
        k, Bp, lb, Xp, lx = self._ptrs(Bts, Xts)
        self._cap_keep = (Bts, Xts)
        _check(lib().ils_batch_capture(self.b, int(bool(refactor)), k, Bp, lb, Xp, lx, int(bool(x0_zero)),
                                       float(tol), int(steps), _stream_ptr(stream)), "ils_batch_capture")

    def run(self, stream=None, allow=(ILS_OK,)):
        """Replay the captured graph; one ils_info per problem."""
        infos = (ils_info * self.count)()
        _check(lib().ils_batch_run(self.b, infos, _stream_ptr(stream)), "ils_batch_run", allow)
        return list(infos)

    def close(self):
        if getattr(self, "b", None):
            lib().ils_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmStartNet:
    """The warm-start perceptron (wraps an ils_mlp).  Tensors are CUDA tensors: theta
    (count, d_in) float32, targets/outputs (count, d_out) float64 (sample-major rows)."""

    def __init__(self, d_in, d_hidden, d_out, seed=0, stream=None):
        h = ctypes.c_void_p()
        _check(lib().ils_mlp_create(ctypes.byref(h), d_in, d_hidden, d_out, seed, _stream_ptr(stream)),
               "ils_mlp_create")
        self.h = h
        self.d_in, self.d_hidden, self.d_out = d_in, d_hidden, d_out

    @property
    def num_params(self):
        return int(lib().ils_mlp_num_params(self.h))

    def get_params(self, out, stream=None):
        return _check(lib().ils_mlp_get_params(self.h, out.data_ptr(), _stream_ptr(stream)), "ils_mlp_get_params")

    def set_params(self, src, stream=None):
        return _check(lib().ils_mlp_set_params(self.h, src.data_ptr(), _stream_ptr(stream)), "ils_mlp_set_params")

    def loss_grad(self, theta, T, grad, stream=None):
        loss = ctypes.c_double()
        _check(lib().ils_mlp_loss_grad(self.h, theta.shape[0], theta.data_ptr(), T.data_ptr(), ctypes.byref(loss),
                                       grad.data_ptr(), _stream_ptr(stream)), "ils_mlp_loss_grad")
        return loss.value

    def train(self, theta, T, epochs, batch=256, lr=1e-3, stream=None):
        loss = ctypes.c_double()
        _check(lib().ils_mlp_train(self.h, theta.shape[0], theta.data_ptr(), T.data_ptr(), epochs, batch, lr,
                                   ctypes.byref(loss), _stream_ptr(stream)), "ils_mlp_train")
        return loss.value

    def forward(self, theta, X, bf16=True, stream=None):
        return _check(lib().ils_mlp_forward(self.h, theta.shape[0], theta.data_ptr(), X.data_ptr(), X.stride(0),
                                            int(bool(bf16)), _stream_ptr(stream)), "ils_mlp_forward")

    def solve(self, solver, theta, Bt, Xt, tol=1e-12, stream=None, allow=(ILS_OK,)):
        """ils_solve_param: x0 = net(theta), then the solver's iteration."""
        k = Bt.shape[0]
        bp, ldb = _colmajor_ptr(Bt, solver.m, k)
        xp, ldx = _colmajor_ptr(Xt, solver.n, k)
        info = ils_info()
        code = lib().ils_solve_param(solver.h, self.h, k, theta.data_ptr(), bp, ldb, xp, ldx, float(tol),
                                     ctypes.byref(info), _stream_ptr(stream))
        _check(code, "ils_solve_param", allow)
        return info

    def close(self):
        if getattr(self, "h", None):
            lib().ils_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
