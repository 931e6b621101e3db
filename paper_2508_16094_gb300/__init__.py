"""GB300-native pivoting-free interior-point solver (arXiv 2508.16094).

Thin ctypes binding of the C ABI in ``include/gb300_ipm.h``: argument
marshalling only, every step of the method runs in ``libgb300ipm.so``. PyTorch
provides device memory (the workspace and the vectors) and the stream.

There is no CPU fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["IpmError", "IpmContext", "Options", "load", "build", "lib_path",
           "IPM_FP64", "IPM_FP32", "IPM_TF32", "IPM_BF16", "IPM_TF32X3",
           "IPM_REFINE_NONE", "IPM_REFINE_IR", "IPM_REFINE_PCG", "IPM_FORM_PRIMAL",
           "IPM_FORM_DUAL", "IPM_FORM_AUGMENTED"]

IPM_FP64, IPM_FP32, IPM_TF32, IPM_BF16, IPM_TF32X3 = 0, 1, 2, 3, 4
IPM_REFINE_NONE, IPM_REFINE_IR, IPM_REFINE_PCG = 0, 1, 2
IPM_FORM_PRIMAL, IPM_FORM_DUAL, IPM_FORM_AUGMENTED = 0, 1, 2
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_CUDA", 4: "ERR_NOMEM", 5: "ERR_NOT_SPD",
          6: "ERR_NUMERIC", 7: "ERR_MAXITER", 8: "ERR_TIMEOUT", 9: "ERR_STALL",
          10: "ERR_UNSUPPORTED"}
EXPORTED = ["ipm_default_options", "ipm_create", "ipm_set_options", "kkt_analyze", "ipm_set_workspace",
            "kkt_assemble", "kkt_factor", "kkt_solve", "ipm_solve", "ipm_newton_direction",
            "kkt_symbolic_export", "kkt_export_assembled", "kkt_factor_entries",
            "ipm_last_perturbed", "kkt_time_kernel", "kkt_test_solve_timeout", "ipm_kernel_launches", "kkt_solve_noalloc",
            "kkt_solve_noalloc_capacity", "ipm_mpc_workspace_bytes", "ipm_mpc_prepare",
            "ipm_solve_batched", "ipm_mpc_autotune", "ipm_learned_param_count",
            "ipm_learned_weights", "ipm_learned_sample", "ipm_learned_loss_grad",
            "ipm_learned_train", "ipm_symbolic_batched_workspace", "ipm_symbolic_batched",
            "ipm_grid_nlp_sizes", "ipm_grid_nlp_pattern",
            "ipm_solve_grid_nlp", "ipm_create_pattern", "ipm_solve_problem", "ipm_solve_nlp",
            "ipm_last_error", "ipm_destroy"]


class IpmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Options(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("tol", C.c_double), ("delta_p", C.c_double),
                ("delta_d", C.c_double), ("precision", C.c_int32), ("storage_fp64", C.c_int32),
                ("refine", C.c_int32), ("ir_max", C.c_int32), ("ir_tol", C.c_double),
                ("pcg_max", C.c_int32), ("fallback_fp64", C.c_int32), ("accept_tol", C.c_double),
                ("verbose", C.c_int32), ("warm_start", C.c_int32), ("learned", C.c_int32),
                ("learned_probes", C.c_int32), ("learned_pcg_max", C.c_int32),
                ("formulation", C.c_int32), ("cg_escalate", C.c_int32),
                ("fp64_tc", C.c_int32)]


class SymbolicInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m_tot", C.c_int64), ("nnz_k", C.c_int64),
                ("nnz_l", C.c_int64), ("nsuper", C.c_int32), ("nlevels", C.c_int32),
                ("max_front", C.c_int32), ("max_ncol", C.c_int32), ("flops", C.c_double),
                ("factor_entries", C.c_int64), ("update_entries", C.c_int64),
                ("workspace_bytes", C.c_int64)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("used_pcg", C.c_int32), ("rel_residual", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("factorizations", C.c_int32),
                ("regularizations", C.c_int32), ("refine_steps", C.c_int32),
                ("pcg_steps", C.c_int32), ("fp64_fallbacks", C.c_int32),
                ("perturbed_pivots", C.c_int32), ("objective", C.c_double), ("kkt", C.c_double),
                ("primal_res", C.c_double), ("dual_res", C.c_double), ("compl_res", C.c_double),
                ("mu", C.c_double), ("worst_rel_residual", C.c_double),
                ("time_total_ms", C.c_double), ("time_assemble_ms", C.c_double),
                ("time_factor_ms", C.c_double), ("time_solve_ms", C.c_double),
                ("time_other_ms", C.c_double), ("learned_skips", C.c_int32),
                ("learned_pcg_steps", C.c_int32), ("fp64_tc_rechecks", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load() -> C.CDLL:
    """Load libgb300ipm.so (built in-tree by ``build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"{_build.LIB} is missing: run paper_2508_16094_gb300.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(_build.LIB)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "ipm_default_options": (None, [P]),
        "ipm_create": (I32, [I32, I32, P, P, P, P, P, P, P, P, P]),
        "ipm_set_options": (I32, [P, P]),
        "kkt_analyze": (I32, [P, P, P]),
        "ipm_set_workspace": (I32, [P, P, C.c_size_t]),
        "kkt_assemble": (I32, [P, P, P, P, D]),
        "kkt_factor": (I32, [P, I32, P]),
        "kkt_solve": (I32, [P, P, P, I32, I32, P]),
        "ipm_solve": (I32, [P, P, P, P, P, P, P, P, P]),
        "ipm_newton_direction": (I32, [P] * 12),
        "kkt_symbolic_export": (I32, [P] * 9),
        "kkt_export_assembled": (I32, [P, P]),
        "kkt_factor_entries": (I32, [P, I64, P, P, P]),
        "ipm_last_perturbed": (I32, [P]),
        "kkt_time_kernel": (I32, [P, I32, I32, P]),
        "kkt_test_solve_timeout": (I32, [P, C.c_uint32, I32]),
        "ipm_kernel_launches": (I64, []),
        "kkt_solve_noalloc": (I32, [P, P, P]),
        "kkt_solve_noalloc_capacity": (I64, []),
        "ipm_mpc_workspace_bytes": (I32, [P, P]),
        "ipm_learned_param_count": (I32, []),
        "ipm_learned_weights": (I32, [P, P, P]),
        "ipm_learned_sample": (I32, [P] * 8),
        "ipm_learned_loss_grad": (I32, [P] * 6),
        "ipm_learned_train": (I32, [P, P, P, P, C.c_float, I32, P]),
        "ipm_mpc_prepare": (I32, [P, P, C.c_size_t, P]),
        "ipm_solve_batched": (I32, [P, P, P, C.c_size_t, D, I32, P, P, P, P, P, P]),
        "ipm_mpc_autotune": (I32, [P, P, C.c_size_t, D, I32, P, P, P, P, P, P, P, P]),
        "ipm_symbolic_batched_workspace": (I32, [P, P]),
        "ipm_symbolic_batched": (I32, [P, P, C.c_size_t, P, P, P, P, P, P]),
        "ipm_grid_nlp_sizes": (I32, [P, P, P, P]),
        "ipm_grid_nlp_pattern": (I32, [P] * 7),
        "ipm_solve_grid_nlp": (I32, [P] * 7),
        "ipm_create_pattern": (I32, [I32, I32, P, P, P, P]),
        "ipm_solve_problem": (I32, [P, P, P, P, P, P]),
        "ipm_solve_nlp": (I32, [P, P, P, P, P, P]),
        "ipm_last_error": (C.c_char_p, [P]),
        "ipm_destroy": (None, [P]),
    }
    for name, (rt, args) in sig.items():
        f = getattr(lib, name)
        f.restype = rt
        f.argtypes = args
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().ipm_kernel_launches())


def default_options(**kw) -> Options:
    o = Options()
    load().ipm_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _np(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _hp(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dp(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class PatternDesc(C.Structure):
    """ipm_pattern (host pointers)."""
    _fields_ = [("j_rowptr", C.c_void_p), ("j_col", C.c_void_p), ("w_colptr", C.c_void_p),
                ("w_row", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p)]


class ProblemDesc(C.Structure):
    """ipm_problem (device pointers; nlp: host ipm_grid_nlp; fns: host ipm_nlp)."""
    _fields_ = [("kind", C.c_int32), ("d_jvals", C.c_void_p), ("d_b", C.c_void_p),
                ("d_c", C.c_void_p), ("d_wvals", C.c_void_p), ("nlp", C.c_void_p),
                ("d_ut", C.c_void_p), ("fns", C.c_void_p)]


NLP_EVAL = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                       C.c_void_p, C.c_void_p)
NLP_HESS = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)


class NlpDesc(C.Structure):
    """ipm_nlp: the evaluation callbacks of a nonlinear problem."""
    _fields_ = [("user", C.c_void_p), ("eval", NLP_EVAL), ("hess", NLP_HESS)]


def device_view(ptr, count: int):
    """A float64 CUDA tensor aliasing `count` doubles of device memory at ptr
    (no copy), for the callbacks of ipm_solve_nlp."""
    import torch

    class _Dev:
        pass

    d = _Dev()
    d.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                  "data": (int(ptr or 0), False), "version": 3}
    return torch.as_tensor(d, device="cuda")


def ipm_create_pattern(n, m, j_rowptr, j_col, l=None, u=None, w_colptr=None, w_row=None,
                       options: "Options | None" = None):
    """ipm_create_pattern: returns the raw context handle (c_void_p) and the
    host arrays it was built from; release it with ipm_destroy."""
    lib = load()
    keep = [_np(j_rowptr, np.int64), _np(j_col, np.int32), _np(w_colptr, np.int64),
            _np(w_row, np.int32), _np(l, np.float64), _np(u, np.float64)]
    p = PatternDesc(*[_hp(a) for a in keep])
    o = options if options is not None else default_options()
    h = C.c_void_p()
    st = lib.ipm_create_pattern(int(n), int(m), C.byref(p), C.byref(o), None, C.byref(h))
    if st != 0:
        raise IpmError(st, "")
    return h, keep


class IpmContext:
    """One solver context; methods are named after the C entry points they call."""

    def __init__(self, n, m, j_rowptr, j_col, l=None, u=None, w_colptr=None, w_row=None,
                 options: Options | None = None, stream=None):
        lib = load()
        self._lib = lib
        self.n, self.m = int(n), int(m)
        self.options = options if options is not None else default_options()
        self._keep = [_np(j_rowptr, np.int64), _np(j_col, np.int32), _np(w_colptr, np.int64),
                      _np(w_row, np.int32), _np(l, np.float64), _np(u, np.float64)]
        h = C.c_void_p()
        st = self._keep
        self._check(lib.ipm_create(self.n, self.m, _hp(st[0]), _hp(st[1]), _hp(st[2]), _hp(st[3]),
                                   _hp(st[4]), _hp(st[5]), C.byref(self.options),
                                   C.c_void_p(stream) if stream else None, C.byref(h)), None)
        self.handle = h
        self.info: SymbolicInfo | None = None
        self.workspace = None
        lf = np.isfinite(st[4]).sum() if st[4] is not None else 0
        uf = np.isfinite(st[5]).sum() if st[5] is not None else 0
        self.m_tot = self.m + int(lf) + int(uf)

    def _check(self, status, handle="self"):
        if status != 0:
            h = self.handle if handle == "self" else None
            msg = self._lib.ipm_last_error(h).decode() if h else ""
            raise IpmError(status, msg)
        return status

    # --- C entry points -----------------------------------------------------
    def ipm_set_options(self, options: Options | None = None, **kw):
        """Push options to the library (the context keeps its own copy)."""
        o = Options()
        C.pointer(o)[0] = options if options is not None else self.options
        for k, v in kw.items():
            setattr(o, k, v)
        self._check(self._lib.ipm_set_options(self.handle, C.byref(o)))
        self.options = o

    def kkt_analyze(self, perm=None) -> SymbolicInfo:
        info = SymbolicInfo()
        p = _np(perm, np.int32)
        self._check(self._lib.kkt_analyze(self.handle, _hp(p), C.byref(info)))
        self.info = info
        return info

    def ipm_set_workspace(self, buf=None):
        """Hand over a device buffer (torch uint8 tensor); allocates one if None."""
        import torch
        if buf is None:
            buf = torch.empty(int(self.info.workspace_bytes) + 256, dtype=torch.uint8, device="cuda")
        self.workspace = buf
        self._check(self._lib.ipm_set_workspace(self.handle, C.c_void_p(buf.data_ptr()),
                                                buf.numel()))
        return buf

    def kkt_assemble(self, jvals, D, delta_p, wvals=None):
        self._check(self._lib.kkt_assemble(self.handle, _dp(wvals), _dp(jvals), _dp(D),
                                           float(delta_p)))

    def kkt_factor(self, precision=IPM_FP64, raise_on_error=True):
        bad = C.c_int32(-1)
        st = self._lib.kkt_factor(self.handle, int(precision), C.byref(bad))
        if raise_on_error:
            self._check(st)
        return st, bad.value

    def kkt_solve(self, b, x, refine=IPM_REFINE_IR, raise_on_error=True) -> SolveInfo:
        """b, x: one right-hand side (length n) or several stored one after
        the other (n * nrhs entries, e.g. a contiguous (nrhs, n) tensor)."""
        info = SolveInfo()
        nsys = self.kkt_order()
        if b.numel() != x.numel() or b.numel() % nsys != 0 or b.numel() == 0:
            raise ValueError("b and x must hold nrhs * n entries")
        st = self._lib.kkt_solve(self.handle, _dp(b), _dp(x), b.numel() // nsys, int(refine),
                                 C.byref(info))
        if raise_on_error:
            self._check(st)
        return info

    def ipm_solve(self, jvals, b, c, x, s, lam, wvals=None, raise_on_error=False) -> Result:
        res = Result()
        st = self._lib.ipm_solve(self.handle, _dp(jvals), _dp(b), _dp(c), _dp(wvals), _dp(x),
                                 _dp(s), _dp(lam), C.byref(res))
        if raise_on_error:
            self._check(st)
        return res

    def ipm_solve_problem(self, x, s, lam, jvals=None, b=None, c=None, wvals=None, nlp=None,
                          ut=None, raise_on_error=False) -> Result:
        """ipm_solve_problem: an LP/QP (jvals, b, c, wvals) or, with nlp (an
        ipm_grid_nlp struct) and ut, the grid NLP."""
        p = ProblemDesc()
        if nlp is None:
            p.kind, p.d_jvals, p.d_b, p.d_c, p.d_wvals = 0, _dp(jvals), _dp(b), _dp(c), _dp(wvals)
        else:
            p.kind, p.nlp, p.d_ut = 1, C.cast(C.pointer(nlp), C.c_void_p), _dp(ut)
        res = Result()
        st = self._lib.ipm_solve_problem(self.handle, C.byref(p), _dp(x), _dp(s), _dp(lam),
                                         C.byref(res))
        if raise_on_error:
            self._check(st)
        return res

    def ipm_solve_nlp(self, eval_fn, hess_fn, x, s, lam, raise_on_error=False) -> Result:
        """ipm_solve_nlp with Python callbacks on torch views of the device
        arrays: eval_fn(x, f, grad, g, jvals) fills f (1), grad (n), g (m general
        rows) and jvals (nnz(J)) at x; hess_fn(x, lam, wvals) fills wvals
        (nnz(W)) at x, lam (m_tot; the first m entries are the general rows').
        A callback that raises ends the solve with IPM_ERR_NUMERIC."""
        n, m, m_tot = self.n, self.m, self.m_tot
        nnz_j = len(self._keep[1]) if self._keep[1] is not None else 0
        nnz_w = len(self._keep[3]) if self._keep[3] is not None else 0

        def _eval(user, px, pf, pg, pgr, pjv, stream):
            try:
                eval_fn(device_view(px, n), device_view(pf, 1), device_view(pg, n),
                        device_view(pgr, m), device_view(pjv, nnz_j))
                return 0
            except Exception:  # reported to the solver as a failed evaluation
                return 1

        def _hess(user, px, plam, pw, stream):
            try:
                hess_fn(device_view(px, n), device_view(plam, m_tot), device_view(pw, nnz_w))
                return 0
            except Exception:
                return 1

        fns = NlpDesc(None, NLP_EVAL(_eval), NLP_HESS(_hess))
        res = Result()
        st = self._lib.ipm_solve_nlp(self.handle, C.byref(fns), _dp(x), _dp(s), _dp(lam),
                                     C.byref(res))
        if raise_on_error:
            self._check(st)
        return res

    def ipm_newton_direction(self, jvals, b, c, x, s, lam, w, dx, ds, dl, wvals=None):
        self._check(self._lib.ipm_newton_direction(self.handle, _dp(jvals), _dp(b), _dp(c),
                                                   _dp(wvals), _dp(x), _dp(s), _dp(lam), _dp(w),
                                                   _dp(dx), _dp(ds), _dp(dl)))

    def kkt_order(self) -> int:
        """Order of the matrix the context factors (n, m or n + m by formulation)."""
        return int(self.info.n) if self.info is not None else self.n

    def kkt_symbolic_export(self) -> dict:
        n, ns = self.kkt_order(), self.info.nsuper
        out = dict(perm=np.empty(n, np.int32), parent=np.empty(n, np.int32),
                   colcount=np.empty(n, np.int32), super=np.empty(ns + 1, np.int32),
                   sparent=np.empty(ns, np.int32), slevel=np.empty(ns, np.int32),
                   srp=np.empty(ns + 1, np.int64))
        self._check(self._lib.kkt_symbolic_export(self.handle, *[_hp(out[k]) for k in
                                                                 ["perm", "parent", "colcount",
                                                                  "super", "sparent", "slevel",
                                                                  "srp"]], None))
        out["sri"] = np.empty(int(out["srp"][-1]), np.int32)
        self._check(self._lib.kkt_symbolic_export(self.handle, None, None, None, None, None,
                                                  None, None, _hp(out["sri"])))
        return out

    def kkt_export_assembled(self) -> np.ndarray:
        out = np.empty(int(self.info.nnz_k), np.float64)
        self._check(self._lib.kkt_export_assembled(self.handle, _hp(out)))
        return out

    def kkt_factor_entries(self, rows, cols) -> np.ndarray:
        r = _np(rows, np.int32)
        c = _np(cols, np.int32)
        out = np.empty(len(r), np.float64)
        self._check(self._lib.kkt_factor_entries(self.handle, len(r), _hp(r), _hp(c), _hp(out)))
        return out

    def kkt_solve_noalloc(self, b, x, raise_on_error=True) -> int:
        """Factor-only solve whose working vectors sit in the library's static
        device array (no device allocation; see the header for its limits)."""
        st = self._lib.kkt_solve_noalloc(self.handle, _dp(b), _dp(x))
        if raise_on_error:
            self._check(st)
        return st

    # --- learned correction ---------------------------------------------------
    def ipm_learned_weights(self, set_to=None) -> np.ndarray:
        n = int(self._lib.ipm_learned_param_count())
        out = np.empty(n, np.float32)
        inp = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float32)
        self._check(self._lib.ipm_learned_weights(self.handle, _hp(out), _hp(inp)))
        return out

    def ipm_learned_sample(self, jvals, x, s, lam, z, feat, w):
        self._check(self._lib.ipm_learned_sample(self.handle, _dp(jvals), _dp(x), _dp(s), _dp(lam),
                                                 _dp(z), _dp(feat), _dp(w)))

    def ipm_learned_loss_grad(self, feat, z, w):
        loss = C.c_double()
        grad = np.empty(int(self._lib.ipm_learned_param_count()), np.float32)
        self._check(self._lib.ipm_learned_loss_grad(self.handle, _dp(feat), _dp(z), _dp(w),
                                                    C.byref(loss), _hp(grad)))
        return loss.value, grad

    def ipm_learned_train(self, feat, z, w, lr=1e-3, steps=1) -> float:
        loss = C.c_double()
        self._check(self._lib.ipm_learned_train(self.handle, _dp(feat), _dp(z), _dp(w),
                                                C.c_float(lr), int(steps), C.byref(loss)))
        return loss.value

    def kkt_time_kernel(self, kernel: int, reps: int = 3) -> float:
        """Milliseconds per launch of one library kernel (0 assembly,
        1 persistent FP32 solve, 2 FP64 level solve) on the current data."""
        ms = C.c_double()
        self._check(self._lib.kkt_time_kernel(self.handle, int(kernel), int(reps), C.byref(ms)))
        return ms.value

    def kkt_test_solve_timeout(self, spins: int, withheld_task: int = 0):
        """Make the next persistent solve's bounded waits run out: every wait
        polls at most ``spins`` times and the task at position
        ``withheld_task`` of the solve's task order is abandoned."""
        self._check(self._lib.kkt_test_solve_timeout(self.handle, int(spins), int(withheld_task)))

    def ipm_last_perturbed(self) -> int:
        return int(self._lib.ipm_last_perturbed(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ipm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MpcBatch(C.Structure):
    _fields_ = [("count", C.c_int32), ("h_T", C.c_void_p), ("d_A", C.c_void_p),
                ("d_B", C.c_void_p), ("d_Q", C.c_void_p), ("d_R", C.c_void_p),
                ("d_x0", C.c_void_p), ("u_max", C.c_double), ("x_max", C.c_double)]


class MpcConfig(C.Structure):
    _fields_ = [("precision", C.c_int32), ("instances_per_cta", C.c_int32), ("ctas", C.c_int32)]


class BatchedMPC:
    """Batched MPC QPs (ipm_mpc_* entry points). ``mb`` holds numpy arrays
    T, A, B, Q, R, x0 (stacked over instances) and the box bounds."""

    def __init__(self, mb, stream=None):
        import torch
        lib = load()
        self._lib = lib
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        self.T = np.ascontiguousarray(mb.T, dtype=np.int32)
        self.count = len(self.T)
        self.total_stages = int(self.T.sum())
        self._t = [dev(mb.A), dev(mb.B), dev(mb.Q), dev(mb.R), dev(mb.x0)]
        self.batch = MpcBatch(self.count, _hp(self.T), *[C.c_void_p(t.data_ptr()) for t in self._t],
                              float(mb.u_max), float(mb.x_max))
        nb = C.c_size_t()
        self._check(lib.ipm_mpc_workspace_bytes(C.byref(self.batch), C.byref(nb)))
        self.work = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        self.wptr = (self.work.data_ptr() + 255) // 256 * 256
        self.wbytes = nb.value
        self.stream = stream
        self._check(lib.ipm_mpc_prepare(C.byref(self.batch), C.c_void_p(self.wptr), self.wbytes,
                                        C.c_void_p(stream) if stream else None))
        self.z = torch.empty(self.total_stages * 16, dtype=torch.float64, device="cuda")
        self.obj = torch.empty(self.count, dtype=torch.float64, device="cuda")
        self.kkt = torch.empty(self.count, dtype=torch.float64, device="cuda")
        self.iters = torch.empty(self.count, dtype=torch.int32, device="cuda")
        self.status = torch.empty(self.count, dtype=torch.int32, device="cuda")

    @staticmethod
    def _check(st):
        if st != 0:
            raise IpmError(st, "batched MPC call failed")

    def ipm_solve_batched(self, precision=IPM_FP64, instances_per_cta=8, ctas=0, tol=1e-6,
                          max_iter=100, stream=None):
        cfg = MpcConfig(precision, instances_per_cta, ctas)
        st = stream if stream is not None else self.stream
        self._check(self._lib.ipm_solve_batched(
            C.byref(self.batch), C.byref(cfg), C.c_void_p(self.wptr), self.wbytes, float(tol),
            int(max_iter), C.c_void_p(st) if st else None, _dp(self.z), _dp(self.obj),
            _dp(self.kkt), _dp(self.iters), _dp(self.status)))

    def ipm_mpc_autotune(self, precision=IPM_FP64, tol=1e-6, max_iter=100):
        cfg = MpcConfig(precision, 8, 0)
        ms = (C.c_float * 16)()
        self._check(self._lib.ipm_mpc_autotune(
            C.byref(self.batch), C.c_void_p(self.wptr), self.wbytes, float(tol), int(max_iter),
            C.c_void_p(self.stream) if self.stream else None, _dp(self.z), _dp(self.obj),
            _dp(self.kkt), _dp(self.iters), _dp(self.status), C.byref(cfg), ms))
        return cfg, list(ms)


# --- symbolic analysis of batched patterns on the GPU ----------------------------
class PatternBatch(C.Structure):
    _fields_ = [("count", C.c_int32), ("h_n", C.c_void_p), ("h_m", C.c_void_p),
                ("h_nnz", C.c_void_p), ("d_rowptr", C.c_void_p), ("d_col", C.c_void_p),
                ("d_perm", C.c_void_p)]


def symbolic_batched(patterns, perms=None, stream=None):
    """ipm_symbolic_batched over a list of (n, rowptr, col) host patterns (CSR
    of J) and optional orderings (new -> old). Returns (post, parent, colcount,
    sstart) as lists of numpy arrays, one per pattern, and the launch's device
    time in milliseconds (CUDA events around the call)."""
    import torch
    lib = load()
    cnt = len(patterns)
    h_n = np.array([p[0] for p in patterns], np.int32)
    h_m = np.array([len(p[1]) - 1 for p in patterns], np.int32)
    h_nnz = np.array([int(p[1][-1]) for p in patterns], np.int64)
    offs = np.concatenate([[0], np.cumsum(h_nnz)])[:-1]
    rp = np.concatenate([np.asarray(p[1], np.int64) + o for p, o in zip(patterns, offs)])
    cl = np.concatenate([np.asarray(p[2], np.int32) for p in patterns]) if h_nnz.sum() else np.zeros(1, np.int32)
    d_rp = torch.as_tensor(rp, device="cuda")
    d_cl = torch.as_tensor(cl, device="cuda")
    d_pm = None
    if perms is not None:
        d_pm = torch.as_tensor(np.concatenate([np.asarray(q, np.int32) for q in perms]), device="cuda")
    b = PatternBatch(cnt, _hp(h_n), _hp(h_m), _hp(h_nnz), C.c_void_p(d_rp.data_ptr()),
                     C.c_void_p(d_cl.data_ptr()), C.c_void_p(d_pm.data_ptr()) if d_pm is not None else None)
    nb = C.c_size_t()
    st = lib.ipm_symbolic_batched_workspace(C.byref(b), C.byref(nb))
    if st != 0:
        raise IpmError(st, "symbolic batch workspace")
    work = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
    wptr = (work.data_ptr() + 255) // 256 * 256
    N = int(h_n.sum())
    outs = [torch.empty(max(N, 1), dtype=torch.int32, device="cuda") for _ in range(4)]
    bad = C.c_int32(-1)
    s = torch.cuda.current_stream() if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    st = lib.ipm_symbolic_batched(C.byref(b), C.c_void_p(wptr), nb.value, C.c_void_p(s.cuda_stream),
                                  *[C.c_void_p(t.data_ptr()) for t in outs], C.byref(bad))
    e1.record(s)
    torch.cuda.synchronize()
    if st != 0:
        raise IpmError(st, f"symbolic batch: pattern {bad.value}")
    host = [t.cpu().numpy() for t in outs]
    cuts = np.cumsum(h_n)[:-1]
    return [np.split(h, cuts) for h in host], e0.elapsed_time(e1)


# --- grid NLP -----------------------------------------------------------------
class GridNlpParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("alpha", C.c_double), ("v_lo", C.c_double),
                ("v_hi", C.c_double), ("cubic", C.c_int32), ("v_bounded", C.c_int32)]


def ipm_grid_nlp_pattern(nx, alpha=5e-3, v_lo=-1.0, v_hi=1.0, cubic=1, v_bounded=1) -> dict:
    """Patterns (J CSR, W lower CSC), bounds and sizes of the grid NLP as the
    library evaluates it."""
    lib = load()
    prm = GridNlpParams(int(nx), float(alpha), float(v_lo), float(v_hi), int(cubic), int(v_bounded))
    n, m, nnz = C.c_int32(), C.c_int32(), C.c_int64()
    st = lib.ipm_grid_nlp_sizes(C.byref(prm), C.byref(n), C.byref(m), C.byref(nnz))
    if st != 0:
        raise IpmError(st, "invalid grid NLP parameters")
    out = dict(params=prm, n=n.value, m=m.value, rowptr=np.empty(m.value + 1, np.int64),
               col=np.empty(nnz.value, np.int32), wp=np.empty(n.value + 1, np.int64),
               wi=np.empty(n.value, np.int32), l=np.empty(n.value), u=np.empty(n.value))
    st = lib.ipm_grid_nlp_pattern(C.byref(prm), *[_hp(out[k]) for k in
                                                  ("rowptr", "col", "wp", "wi", "l", "u")])
    if st != 0:
        raise IpmError(st, "grid NLP pattern")
    return out


class GridNLP:
    """Context for the grid NLP: created with the library's patterns, analysed
    with the given ordering; ipm_solve_grid_nlp runs the method."""

    def __init__(self, nx, perm=None, alpha=5e-3, v_lo=-1.0, v_hi=1.0, cubic=1, v_bounded=1,
                 options: Options | None = None):
        self.pat = ipm_grid_nlp_pattern(nx, alpha, v_lo, v_hi, cubic, v_bounded)
        pt = self.pat
        self.ctx = IpmContext(pt["n"], pt["m"], pt["rowptr"], pt["col"], pt["l"], pt["u"],
                              pt["wp"], pt["wi"], options=options)
        self.info = self.ctx.kkt_analyze(perm)
        self.ctx.ipm_set_workspace()

    def ipm_solve_grid_nlp(self, ut, x, s, lam, raise_on_error=False) -> Result:
        res = Result()
        st = self.ctx._lib.ipm_solve_grid_nlp(self.ctx.handle, C.byref(self.pat["params"]), _dp(ut),
                                              _dp(x), _dp(s), _dp(lam), C.byref(res))
        if raise_on_error:
            self.ctx._check(st)
        return res
