"""ctypes binding of the opevo C ABI (include/opevo.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
buffers for the kernel-level calls are torch CUDA tensors (PyTorch provides
device memory and streams); host buffers are numpy arrays.  The binding fails
loudly when ``libopevo.so`` is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libopevo.so")

OP_OK, OP_ERR_ARG, OP_ERR_CUDA, OP_ERR_NOTSPD, OP_ERR_DIVERGED, OP_ERR_TIMEOUT, OP_ERR_OOM, \
    OP_ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7
OP_FP64, OP_FP32, OP_MIX_TF32, OP_MIX_BF16X3, OP_MIX_BF16 = 0, 1, 2, 3, 4
OP_STOP_RESIDUAL, OP_STOP_ERR_E, OP_STOP_STEPS = 0, 1, 2
OP_EIG_RITZ, OP_EIG_PAPER = 0, 1
PRECS = {"fp64": OP_FP64, "fp32": OP_FP32, "mix_tf32": OP_MIX_TF32, "mix_bf16x3": OP_MIX_BF16X3,
         "mix_bf16": OP_MIX_BF16}
STATUS_NAMES = {0: "OP_OK", -1: "OP_ERR_ARG", -2: "OP_ERR_CUDA", -3: "OP_ERR_NOTSPD",
                -4: "OP_ERR_DIVERGED", -5: "OP_ERR_TIMEOUT", -6: "OP_ERR_OOM",
                -7: "OP_ERR_STATE"}


class OpProblem(C.Structure):
    _fields_ = [("dim", C.c_int), ("shape", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("p", C.c_int), ("sigma", C.c_double),
                ("tau", C.c_double), ("prec", C.c_int), ("cg_rtol", C.c_double),
                ("cg_max_iter", C.c_int), ("check_every", C.c_int), ("adapt_every", C.c_int),
                ("cg_precond", C.c_int), ("flow", C.c_int), ("fp64_gemm", C.c_int),
                ("step1", C.c_int)]


class OpStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("last_cg_iters", C.c_int), ("cg_iters", C.c_longlong),
                ("energy", C.c_double), ("err_E", C.c_double), ("residual", C.c_double),
                ("g_residual", C.c_double), ("orth", C.c_double), ("sigma", C.c_double),
                ("tau", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OpShardStats(C.Structure):
    _fields_ = [("slabs", C.c_int), ("halo_copies", C.c_longlong), ("halo_bytes", C.c_longlong),
                ("reductions", C.c_longlong), ("reduction_bytes", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OpnetConfig(C.Structure):
    _fields_ = [("N", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("p", C.c_int),
                ("width", C.c_int * 3), ("stream", C.c_void_p)]


class OpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libopevo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, sz, i32, f64 = C.c_void_p, C.c_size_t, C.c_int, C.c_double
    P = C.POINTER
    sigs = {
        "op_version": (C.c_char_p, []),
        "op_last_error": (C.c_char_p, []),
        "op_kernel_launches": (C.c_longlong, []),
        "op_init": (i32, [P(vp), P(OpProblem), P(f64), P(f64), vp]),
        "op_init_device": (i32, [P(vp), P(OpProblem), vp, vp, vp]),
        "op_init_seeded": (i32, [P(vp), P(OpProblem), P(f64), C.c_ulonglong, vp]),
        "op_gaussian_block": (i32, [C.c_ulonglong, C.c_longlong, i32, vp, vp]),
        "op_step": (i32, [vp, i32, P(OpStats)]),
        "op_solve": (i32, [vp, f64, i32, i32, P(OpStats)]),
        "op_step_sharded": (i32, [vp, i32, i32, P(OpStats), P(OpShardStats)]),
        "op_energy": (i32, [vp, P(f64)]),
        "op_residual": (i32, [vp, P(f64)]),
        "op_get_U": (i32, [vp, P(f64)]),
        "op_eigenvalues": (i32, [vp, P(f64), i32]),
        "op_get_stats": (i32, [vp, P(OpStats)]),
        "op_profile_enable": (i32, [vp, i32]),
        "op_profile_kinds": (i32, []),
        "op_profile_name": (C.c_char_p, [i32]),
        "op_profile_read": (i32, [vp, i32, P(f64), P(C.c_longlong)]),
        "op_destroy": (None, [vp]),
        "op_batch_create": (i32, [P(vp), P(vp), i32, i32, vp]),
        "op_batch_set_tiles": (i32, [vp, i32, i32]),
        "op_batch_get_tiles": (i32, [vp, P(i32), P(i32)]),
        "op_batch_autotune": (i32, [vp, C.c_char_p, i32, P(f64)]),
        "op_batch_step": (i32, [vp, i32]),
        "op_batch_solve": (i32, [vp, f64, i32, i32, i32, P(i32)]),
        "op_batch_unfreeze": (i32, [vp]),
        "op_batch_stats": (i32, [vp, i32, P(OpStats), P(i32)]),
        "op_batch_destroy": (None, [vp]),
        "op_apply_H": (i32, [P(OpProblem), i32, vp, f64, vp, vp, vp]),
        "op_cg_solve": (i32, [P(OpProblem), i32, vp, f64, vp, vp, f64, i32, vp, sz, P(i32), vp]),
        "op_cg_workspace": (sz, [P(OpProblem), i32]),
        "op_gram": (i32, [i32, C.c_longlong, i32, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
        "op_gram_workspace": (sz, [i32, C.c_longlong, i32]),
        "op_gram_noalloc": (i32, [i32, C.c_longlong, i32, i32, vp, vp, vp, vp, vp, vp]),
        "op_core": (i32, [i32, i32, i32, f64, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "op_core_workspace": (sz, [i32, i32]),
        "op_core_status": (i32, [vp, vp]),
        "op_update": (i32, [i32, C.c_longlong, i32, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
        "op_update_workspace": (sz, [i32, i32]),
        "op_fp64tc_workspace": (sz, [C.c_longlong, i32]),
        "op_gram_fp64tc": (i32, [C.c_longlong, i32, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
        "op_update_fp64tc": (i32, [C.c_longlong, i32, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
        "op_ws_status": (i32, [vp, vp]),
        "op_get_U_device": (i32, [vp, vp, i32]),
        "op_selftest_bounded_waits": (i32, [P(f64), vp]),
        "op_peak_rate": (i32, [i32, P(f64), vp]),
        "op_checkpoint_size": (sz, [vp]),
        "op_checkpoint": (i32, [vp, vp, sz]),
        "op_restore": (i32, [vp, vp, sz]),
        "opnet_create": (i32, [P(vp), P(OpnetConfig)]),
        "opnet_param_count": (C.c_longlong, [vp]),
        "opnet_layer": (i32, [vp, i32, P(i32), P(i32), P(i32)]),
        "opnet_set_params": (i32, [vp, P(C.c_float), C.c_longlong]),
        "opnet_get_params": (i32, [vp, P(C.c_float), C.c_longlong]),
        "opnet_set_conv": (i32, [vp, i32]),
        "opnet_conv": (i32, [i32, vp, i32, i32, i32, i32, vp, vp, vp, vp, vp]),
        "opnet_conv_dgrad": (i32, [i32, vp, i32, i32, i32, i32, vp, vp, vp]),
        "opnet_forward": (i32, [vp, vp, vp]),
        "opnet_infer": (i32, [vp, vp, vp]),
        "opnet_loss_grad": (i32, [vp, vp, vp, f64, P(f64), P(C.c_float), C.c_longlong]),
        "opnet_train_step": (i32, [vp, vp, vp, f64, f64, f64, f64, f64, P(f64)]),
        "opnet_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != OP_OK:
        raise OpError(status, lib().op_last_error().decode())


def last_error() -> str:
    return lib().op_last_error().decode()


PRECONDS = {"none": 0, "jacobi": 1}
FLOWS = {"g": 0, "l2": 1}
FP64_GEMMS = {"tc": 0, "fma": 1}
STEP1 = {"auto": 0, "cg": 1, "refine": 2}


def make_problem(shape, lo, hi, p, *, prec="fp64", sigma=None, tau=None, cg_rtol=0.0,
                 cg_max_iter=0, check_every=0, adapt_every=0, precond="jacobi",
                 flow="g", fp64_gemm="tc", step1="auto") -> OpProblem:
    pb = OpProblem()
    dim = len(shape)
    pb.dim = dim
    for d in range(3):
        pb.shape[d] = int(shape[d]) if d < dim else 1
        pb.lo[d] = float(lo[d]) if d < dim else 0.0
        pb.hi[d] = float(hi[d]) if d < dim else 1.0
    pb.p = int(p)
    pb.sigma = math.nan if sigma is None else float(sigma)
    pb.tau = math.nan if tau is None else float(tau)
    pb.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    pb.cg_rtol = float(cg_rtol)
    pb.cg_max_iter = int(cg_max_iter)
    pb.check_every = int(check_every)
    pb.adapt_every = int(adapt_every)
    pb.cg_precond = PRECONDS[precond] if isinstance(precond, str) else int(precond)
    pb.flow = FLOWS[flow] if isinstance(flow, str) else int(flow)
    pb.fp64_gemm = FP64_GEMMS[fp64_gemm] if isinstance(fp64_gemm, str) else int(fp64_gemm)
    pb.step1 = STEP1[step1] if isinstance(step1, str) else int(step1)
    return pb


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Solver:
    """A solver context (op_init ... op_destroy) for one eigenproblem.

    prec: "fp64", "fp32", "mix_tf32", "mix_bf16x3" or "mix_bf16" (op_prec).
    precond: the Step-1 CG, "jacobi" (preconditioned with diag(H + sigma)) or "none".
    flow: "g" (the paper's model, Step 1 solving W = (H + sigma)^-1 U) or "l2" (the L2
    gradient flow W = -(H + sigma) U through the exact Cayley step; CFL-limited).
    fp64_gemm: "tc" (FP64 Gram and update as exact digit products on the tensor cores) or
    "fma" (FP64 FMA) for FP64 contexts and every context's set-up (op_fp64_gemm).
    step1: "auto", "cg" or "refine" (FP64 iterative refinement around an FP32 CG; op_step1).
    U0 None: the raw initial block is drawn on the device from `seed` (op_init_seeded,
    the stream of synthetic.gaussian_block(seed, n, p)).
    The remaining keywords are the op_problem fields of the same names.
    """

    def __init__(self, shape, lo, hi, V, U0, p, *, prec="fp64", sigma=None, tau=None,
                 cg_rtol=0.0, cg_max_iter=0, check_every=0, adapt_every=0, precond="jacobi",
                 flow="g", stream=None, device=False, seed=0, fp64_gemm="tc", step1="auto"):
        self.pb = make_problem(shape, lo, hi, p, prec=prec, sigma=sigma, tau=tau,
                               cg_rtol=cg_rtol, cg_max_iter=cg_max_iter, check_every=check_every,
                               adapt_every=adapt_every, precond=precond, flow=flow,
                               fp64_gemm=fp64_gemm, step1=step1)
        self.n = int(np.prod(shape))
        self.p = int(p)
        self._ctx = C.c_void_p()
        L = lib()
        st = _stream_ptr(stream)
        if U0 is None:
            # the raw initial block is drawn on the device from `seed` (op_init_seeded)
            V = np.ascontiguousarray(V, dtype=np.float64)
            assert V.shape == (self.n,)
            check(L.op_init_seeded(C.byref(self._ctx), C.byref(self.pb), _dptr(V),
                                   C.c_ulonglong(int(seed) & 0xFFFFFFFFFFFFFFFF), st))
        elif device:
            # V, U0: torch CUDA tensors (float64, contiguous)
            check(L.op_init_device(C.byref(self._ctx), C.byref(self.pb),
                                   C.c_void_p(V.data_ptr()), C.c_void_p(U0.data_ptr()), st))
        else:
            V = np.ascontiguousarray(V, dtype=np.float64)
            U0 = np.ascontiguousarray(U0, dtype=np.float64)
            assert V.shape == (self.n,) and U0.shape == (self.n, self.p)
            check(L.op_init(C.byref(self._ctx), C.byref(self.pb), _dptr(V), _dptr(U0), st))

    def close(self):
        if self._ctx:
            lib().op_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, nsteps=1) -> dict:
        st = OpStats()
        check(lib().op_step(self._ctx, int(nsteps), C.byref(st)))
        return st.as_dict()

    def step_sharded(self, nslab, nsteps=1):
        """op_step_sharded: `nsteps` steps with the grid split into `nslab` slabs along its
        slowest axis (FP64 contexts).  Returns (stats, communication) dicts."""
        st, comm = OpStats(), OpShardStats()
        check(lib().op_step_sharded(self._ctx, int(nslab), int(nsteps), C.byref(st),
                                    C.byref(comm)))
        return st.as_dict(), comm.as_dict()

    def solve(self, tol, max_steps, stop=OP_STOP_RESIDUAL, raise_on_max=True) -> dict:
        st = OpStats()
        s = lib().op_solve(self._ctx, float(tol), int(max_steps), int(stop), C.byref(st))
        if s != OP_OK and (raise_on_max or s != OP_ERR_STATE):
            check(s)
        d = st.as_dict()
        d["converged"] = s == OP_OK
        return d

    def stats(self) -> dict:
        st = OpStats()
        check(lib().op_get_stats(self._ctx, C.byref(st)))
        return st.as_dict()

    def energy(self) -> float:
        e = C.c_double()
        check(lib().op_energy(self._ctx, C.byref(e)))
        return e.value

    def residual(self) -> float:
        r = C.c_double()
        check(lib().op_residual(self._ctx, C.byref(r)))
        return r.value

    def get_U(self, out=None) -> np.ndarray:
        """U (n x p float64) in host memory; `out`, if given, is filled and returned."""
        U = np.empty((self.n, self.p)) if out is None else out
        assert U.shape == (self.n, self.p)
        check(lib().op_get_U(self._ctx, _dptr(U)))
        return U

    def get_U_device(self, dtype=None):
        """The current U as an n x p torch CUDA tensor (float64 or float32)."""
        import torch
        dtype = dtype or torch.float64
        out = torch.empty(self.n, self.p, dtype=dtype, device="cuda")
        check(lib().op_get_U_device(self._ctx, C.c_void_p(out.data_ptr()),
                                    OP_FP64 if dtype == torch.float64 else OP_FP32))
        return out

    def run_logged(self, nsteps, path, residual_every=10):
        """Advance nsteps steps one at a time and append one JSON line per step to `path`:
        the per-step series of §5 (energy, err_E, ||U^T U - I||_F, the G-residual,
        CG iterations, wall-clock ms) plus the residual r every `residual_every` steps."""
        import json
        import time
        with open(path, "a") as f:
            for k in range(int(nsteps)):
                t = time.perf_counter()
                st = self.step(1)
                row = {"step": st["steps"], "energy": st["energy"], "err_E": st["err_E"],
                       "orth": st["orth"], "g_residual": st["g_residual"],
                       "cg_iters": st["last_cg_iters"], "sigma": st["sigma"], "tau": st["tau"],
                       "ms": 1e3 * (time.perf_counter() - t)}
                if residual_every and st["steps"] % residual_every == 0:
                    row["residual"] = self.residual()
                f.write(json.dumps(row) + "\n")
        return self.stats()

    def checkpoint(self) -> np.ndarray:
        """The context's state (U, W, sigma, tau, statistics) as a host byte array."""
        buf = np.empty(int(lib().op_checkpoint_size(self._ctx)), dtype=np.uint8)
        check(lib().op_checkpoint(self._ctx, buf.ctypes.data_as(C.c_void_p), buf.size))
        return buf

    def restore(self, buf: np.ndarray):
        """Load a state written by checkpoint() of a context of the same size and precision."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().op_restore(self._ctx, buf.ctypes.data_as(C.c_void_p), buf.size))

    def profile(self, enable=True):
        """Enable (and reset) or disable per-kernel event timing."""
        check(lib().op_profile_enable(self._ctx, int(bool(enable))))

    def profile_read(self) -> dict:
        """{kernel group: (total device ms, timed launch groups)} since enabling."""
        L = lib()
        out = {}
        for k in range(L.op_profile_kinds()):
            ms, cnt = C.c_double(), C.c_longlong()
            check(L.op_profile_read(self._ctx, k, C.byref(ms), C.byref(cnt)))
            out[L.op_profile_name(k).decode()] = (ms.value, cnt.value)
        return out

    def eigenvalues(self, kind=OP_EIG_RITZ) -> np.ndarray:
        lam = np.empty(self.p)
        check(lib().op_eigenvalues(self._ctx, _dptr(lam), int(kind)))
        return lam


class Batch:
    """Many FP32 Solver contexts advanced together by graph-captured batched kernels.

    The solvers stay owned by the caller and must outlive the batch; while the batch
    exists they must not be stepped individually."""

    def __init__(self, solvers, cg_iters=12, stream=None):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._ctx.value for s in self.solvers])
        self._b = C.c_void_p()
        check(lib().op_batch_create(C.byref(self._b), arr, len(self.solvers), int(cg_iters),
                                    _stream_ptr(stream)))

    def close(self):
        if self._b:
            lib().op_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_tiles(self, rows_per_item, gram_rows):
        check(lib().op_batch_set_tiles(self._b, int(rows_per_item), int(gram_rows)))

    def tiles(self):
        r, g = C.c_int(), C.c_int()
        check(lib().op_batch_get_tiles(self._b, C.byref(r), C.byref(g)))
        return r.value, g.value

    def autotune(self, cache_path=None, steps_per_trial=2):
        ms = C.c_double()
        path = cache_path.encode() if cache_path else None
        check(lib().op_batch_autotune(self._b, path, int(steps_per_trial), C.byref(ms)))
        return ms.value

    def step(self, nsteps=1):
        check(lib().op_batch_step(self._b, int(nsteps)))

    def solve(self, tol, max_steps, stop=OP_STOP_RESIDUAL, check_every=10, raise_on_max=True):
        nc = C.c_int()
        s = lib().op_batch_solve(self._b, float(tol), int(max_steps), int(stop), int(check_every),
                                 C.byref(nc))
        if s != OP_OK and (raise_on_max or s != OP_ERR_STATE):
            check(s)
        return nc.value

    def unfreeze(self):
        check(lib().op_batch_unfreeze(self._b))

    def stats(self, i):
        st, fr = OpStats(), C.c_int()
        check(lib().op_batch_stats(self._b, int(i), C.byref(st), C.byref(fr)))
        d = st.as_dict()
        d["frozen"] = fr.value
        return d


# ----------------------------------------------------------------------------
# Kernel-level calls on torch CUDA tensors
# ----------------------------------------------------------------------------
def _tptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return OP_FP64
    if t.dtype == torch.float32:
        return OP_FP32
    raise TypeError(f"unsupported dtype {t.dtype}")


def apply_H(shape, lo, hi, V_t, sigma, X, Y=None, stream=None):
    """Y = (H + sigma) X for an n x ld block X (torch CUDA, float32/float64)."""
    import torch
    n, ld = X.shape
    prec = _prec_of(X)
    pb = make_problem(shape, lo, hi, ld, prec=prec)
    if Y is None:
        Y = torch.empty_like(X)
    check(lib().op_apply_H(C.byref(pb), ld, _tptr(V_t), float(sigma), _tptr(X), _tptr(Y),
                           _stream_ptr(stream)))
    return Y


def cg_solve(shape, lo, hi, V_t, sigma, U, W, p, rtol, max_iter=5000, stream=None,
             precond="none"):
    """Step 1 alone (op_cg_solve): W <- (H + sigma)^-1 U by block CG warm-started from
    W, each column to ||u - (H + sigma) w|| <= rtol ||u||.  precond: "none" (plain CG,
    the kernel-level default) or "jacobi" (the Solver default).  Returns the number of
    iterations."""
    import torch
    n, ld = U.shape
    prec = _prec_of(U)
    pb = make_problem(shape, lo, hi, p, prec=prec, precond=precond)
    nbytes = lib().op_cg_workspace(C.byref(pb), ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)
    it = C.c_int()
    check(lib().op_cg_solve(C.byref(pb), ld, _tptr(V_t), float(sigma), _tptr(U), _tptr(W),
                            float(rtol), int(max_iter), _tptr(ws), nbytes, C.byref(it),
                            _stream_ptr(stream)))
    return it.value


def gram(U, W, p, want=("C", "S", "D"), stream=None, prec=None):
    """(C, S, D) = (<W,U>, <W,W>, <U,U>) as ld x ld float64 CUDA tensors.  prec: None (by
    the dtype) or "mix_bf16x3" for FP32 blocks on the BF16 x 3 tensor-core path."""
    import torch
    n, ld = U.shape
    prec = _prec_of(U) if prec is None else PRECS[prec]
    out = {k: (torch.empty(ld, ld, dtype=torch.float64, device=U.device) if k in want else None)
           for k in ("C", "S", "D")}
    nbytes = lib().op_gram_workspace(prec, n, ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)
    st = _stream_ptr(stream)
    check(lib().op_gram(prec, n, p, ld, _tptr(U), _tptr(W), _tptr(out["C"]), _tptr(out["S"]),
                        _tptr(out["D"]), _tptr(ws), nbytes, st))
    check(lib().op_ws_status(_tptr(ws), st))
    return out["C"], out["S"], out["D"]


def gram_noalloc(U, W, p, want=("C", "S", "D"), stream=None):
    """As gram(), through op_gram_noalloc (no device allocation by the library; the
    output matrices are allocated here by torch, as a caller would)."""
    import torch
    n, ld = U.shape
    prec = _prec_of(U)
    out = {k: (torch.empty(ld, ld, dtype=torch.float64, device=U.device) if k in want else None)
           for k in ("C", "S", "D")}
    check(lib().op_gram_noalloc(prec, n, p, ld, _tptr(U), _tptr(W), _tptr(out["C"]),
                                _tptr(out["S"]), _tptr(out["D"]), _stream_ptr(stream)))
    return out["C"], out["S"], out["D"]


def core(Cm, Sm, p, tau, dtype=None, stream=None):
    """Steps 2-3: returns (KU, KW) FP64 and (KU_t, KW_t) in `dtype` (ld x ld CUDA)."""
    import torch
    ld = Cm.shape[0]
    dtype = dtype or torch.float64
    prec = OP_FP64 if dtype == torch.float64 else OP_FP32
    KU = torch.empty(ld, ld, dtype=torch.float64, device=Cm.device)
    KW = torch.empty_like(KU)
    KU_t = torch.empty(ld, ld, dtype=dtype, device=Cm.device)
    KW_t = torch.empty_like(KU_t)
    nbytes = lib().op_core_workspace(p, ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=Cm.device)
    st = _stream_ptr(stream)
    check(lib().op_core(prec, p, ld, float(tau), _tptr(Cm), _tptr(Sm), _tptr(KU), _tptr(KW),
                        _tptr(KU_t), _tptr(KW_t), _tptr(ws), nbytes, st))
    check(lib().op_core_status(_tptr(ws), st))
    return KU, KW, KU_t, KW_t


def update(U, W, KU_t, KW_t, p, out=None, stream=None, prec=None):
    import torch
    n, ld = U.shape
    prec = _prec_of(U) if prec is None else PRECS[prec]
    if out is None:
        out = torch.empty_like(U)
    nbytes = lib().op_update_workspace(prec, ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)
    st = _stream_ptr(stream)
    check(lib().op_update(prec, n, p, ld, _tptr(U), _tptr(W), _tptr(KU_t), _tptr(KW_t),
                          _tptr(out), _tptr(ws), nbytes, st))
    check(lib().op_ws_status(_tptr(ws), st))
    return out


def gram_fp64tc(U, W, p, want=("C", "S", "D"), stream=None):
    """(C, S, D) as gram() for float64 blocks through op_gram_fp64tc (exact digit products
    on the tensor cores).  W may be None when only D is wanted."""
    import torch
    n, ld = U.shape
    out = {k: (torch.empty(ld, ld, dtype=torch.float64, device=U.device) if k in want else None)
           for k in ("C", "S", "D")}
    nbytes = lib().op_fp64tc_workspace(n, ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)
    st = _stream_ptr(stream)
    check(lib().op_gram_fp64tc(n, p, ld, _tptr(U), _tptr(W), _tptr(out["C"]), _tptr(out["S"]),
                               _tptr(out["D"]), _tptr(ws), nbytes, st))
    check(lib().op_ws_status(_tptr(ws), st))
    return out["C"], out["S"], out["D"]


def update_fp64tc(U, W, KU, KW, p, out=None, stream=None):
    """Unew = U KU + W KW for float64 blocks through op_update_fp64tc (W, KW may be None)."""
    import torch
    n, ld = U.shape
    if out is None:
        out = torch.empty_like(U)
    nbytes = lib().op_fp64tc_workspace(n, ld)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)
    st = _stream_ptr(stream)
    check(lib().op_update_fp64tc(n, p, ld, _tptr(U), _tptr(W), _tptr(KU), _tptr(KW), _tptr(out),
                                 _tptr(ws), nbytes, st))
    check(lib().op_ws_status(_tptr(ws), st))
    return out


def net_conv(kind, X, N, taps, W, bias=None, stream=None):
    """One layer of the network's convolution (opnet_conv): X (N^3 x cin) and W
    (taps * cin x cout) float32 CUDA tensors, bias (cout) or None; returns (Z, A)."""
    import torch
    n, cin = X.shape
    cout = W.shape[1]
    Z = torch.empty(n, cout, dtype=torch.float32, device=X.device)
    A = torch.empty_like(Z)
    check(lib().opnet_conv(Net.CONV[kind], C.c_void_p(X.data_ptr()), int(N), int(taps), int(cin),
                           int(cout), C.c_void_p(W.data_ptr()),
                           C.c_void_p(bias.data_ptr() if bias is not None else 0),
                           C.c_void_p(Z.data_ptr()), C.c_void_p(A.data_ptr()),
                           _stream_ptr(stream)))
    return Z, A


def net_conv_dgrad(kind, dZ, N, taps, W, stream=None):
    """The data gradient of one layer (opnet_conv_dgrad): dZ (N^3 x cout) and W
    (taps * cin x cout) float32 CUDA tensors; returns dX (N^3 x cin)."""
    import torch
    n, cout = dZ.shape
    cin = W.shape[0] // taps
    dX = torch.empty(n, cin, dtype=torch.float32, device=dZ.device)
    check(lib().opnet_conv_dgrad(Net.CONV[kind], C.c_void_p(dZ.data_ptr()), int(N), int(taps),
                                 int(cin), int(cout), C.c_void_p(W.data_ptr()),
                                 C.c_void_p(dX.data_ptr()), _stream_ptr(stream)))
    return dX


class Net:
    """The learned warm start (include/opnet.h): a 3-level conv U-Net V -> Y (n x p).

    V and targets are torch CUDA tensors (V: N^3 float64; Ustar: N^3 x p float32 with
    orthonormal columns); parameters move as numpy float32 vectors."""

    def __init__(self, N, lo, hi, p, widths=(24, 48, 96), stream=None):
        cfg = OpnetConfig()
        cfg.N = int(N)
        for d in range(3):
            cfg.lo[d] = float(lo[d])
            cfg.hi[d] = float(hi[d])
            cfg.width[d] = int(widths[d])
        cfg.p = int(p)
        cfg.stream = _stream_ptr(stream).value
        self.N, self.p, self.n = int(N), int(p), int(N) ** 3
        self._net = C.c_void_p()
        check(lib().opnet_create(C.byref(self._net), C.byref(cfg)))
        self.count = int(lib().opnet_param_count(self._net))

    def close(self):
        if self._net:
            lib().opnet_destroy(self._net)
            self._net = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    CONV = {"fp32": 0, "bf16_tc": 1}

    def set_conv(self, kind):
        """Arithmetic of the forward convolutions: "bf16_tc" (tensor cores, the default) or
        "fp32" (CUDA cores)."""
        check(lib().opnet_set_conv(self._net, self.CONV[kind]))

    def layers(self):
        """[(taps, Cin, Cout)] of the 11 layers."""
        out = []
        for i in range(11):
            t, ci, co = C.c_int(), C.c_int(), C.c_int()
            check(lib().opnet_layer(self._net, i, C.byref(t), C.byref(ci), C.byref(co)))
            out.append((t.value, ci.value, co.value))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.count
        check(lib().opnet_set_params(self._net, theta.ctypes.data_as(C.POINTER(C.c_float)),
                                     self.count))

    def get_params(self) -> np.ndarray:
        theta = np.empty(self.count, dtype=np.float32)
        check(lib().opnet_get_params(self._net, theta.ctypes.data_as(C.POINTER(C.c_float)),
                                     self.count))
        return theta

    def forward(self, V):
        import torch
        Y = torch.empty(self.n, self.p, dtype=torch.float32, device=V.device)
        check(lib().opnet_forward(self._net, C.c_void_p(V.data_ptr()), C.c_void_p(Y.data_ptr())))
        return Y

    def infer(self, V):
        """The warm-start block (n x p float64 CUDA tensor) for Solver(..., device=True)."""
        import torch
        U0 = torch.empty(self.n, self.p, dtype=torch.float64, device=V.device)
        check(lib().opnet_infer(self._net, C.c_void_p(V.data_ptr()), C.c_void_p(U0.data_ptr())))
        return U0

    def loss_grad(self, V, Ustar, gamma=0.1, grad=True):
        loss = C.c_double()
        g = np.empty(self.count, dtype=np.float32) if grad else None
        check(lib().opnet_loss_grad(self._net, C.c_void_p(V.data_ptr()),
                                    C.c_void_p(Ustar.data_ptr()), float(gamma), C.byref(loss),
                                    g.ctypes.data_as(C.POINTER(C.c_float)) if grad else None,
                                    self.count))
        return loss.value, g

    def train_step(self, V, Ustar, lr, gamma=0.1, beta1=0.9, beta2=0.999, eps=1e-8) -> float:
        loss = C.c_double()
        check(lib().opnet_train_step(self._net, C.c_void_p(V.data_ptr()),
                                     C.c_void_p(Ustar.data_ptr()), float(gamma), float(lr),
                                     float(beta1), float(beta2), float(eps), C.byref(loss)))
        return loss.value


def gaussian_block(seed, n, p, device=None, stream=None):
    """The raw initial block of op_init_seeded (synthetic.gaussian_block's stream) drawn on
    the device: an n x p float64 CUDA tensor."""
    import torch
    out = torch.empty(n, p, dtype=torch.float64, device=device or "cuda")
    check(lib().op_gaussian_block(C.c_ulonglong(int(seed) & 0xFFFFFFFFFFFFFFFF), int(n), int(p),
                                  _tptr(out), _stream_ptr(stream)))
    return out


PEAKS = {"fp64_fma": 0, "tf32_mma": 1, "bf16_mma": 2, "bf16_mma_n64": 3,
         "bf16_mma_n64_areuse": 4}


def peak_rate(kind, stream=None) -> float:
    """TFLOP/s of the library's own microbenchmark of `kind` (PEAKS) on this device."""
    v = C.c_double()
    check(lib().op_peak_rate(PEAKS[kind], C.byref(v), _stream_ptr(stream)))
    return v.value


def selftest_bounded_waits(stream=None):
    """Make one bounded device wait of each kind run out; returns their durations (s)."""
    secs = (C.c_double * 2)()
    check(lib().op_selftest_bounded_waits(secs, _stream_ptr(stream)))
    return secs[0], secs[1]
