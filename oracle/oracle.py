"""ctypes wrapper of the C oracle (test infrastructure; see the package docstring)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def lib_path() -> str:
    return _SO


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                               "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_SO)
        P = C.c_void_p
        lib.orc_analyze.restype = P
        lib.orc_analyze.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P]
        lib.orc_sym_free.argtypes = [P]
        for name, rt in [("orc_sym_n", C.c_int32), ("orc_sym_nsuper", C.c_int32),
                         ("orc_sym_nnz_korig", C.c_int64), ("orc_sym_nnz_lstruct", C.c_int64),
                         ("orc_sym_nnz_srows", C.c_int64), ("orc_sym_nnz_l", C.c_int64),
                         ("orc_sym_flops", C.c_double)]:
            f = getattr(lib, name)
            f.restype = rt
            f.argtypes = [P]
        lib.orc_sym_export.argtypes = [P] * 13
        lib.orc_assemble.restype = C.c_int
        lib.orc_assemble.argtypes = [P, C.c_int32, P, P, P, P, P, P, P, P, C.c_double, P]
        lib.orc_factor.restype = C.c_int32
        lib.orc_factor.argtypes = [P, P, P]
        lib.orc_solve.argtypes = [P, P, P, P]
        lib.orc_factor_ldlt.restype = C.c_int32
        lib.orc_factor_ldlt.argtypes = [P, P, P, P, P]
        lib.orc_solve_ldlt.argtypes = [P, P, P, P, P]
        lib.orc_kmatvec.argtypes = [P, P, P, P]
        lib.orc_lp_direction.restype = C.c_int32
        lib.orc_lp_direction.argtypes = [P, C.c_int32] + [P] * 11 + [C.c_double, C.c_double,
                                                                     C.c_int32, P, P, P, P, P, P]
        lib.orc_ipm_lp.restype = C.c_int
        lib.orc_ipm_lp.argtypes = [P, C.c_int32] + [P] * 17
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


@dataclass
class OracleSymbolic:
    """Symbolic analysis result (final numbering = given ordering + etree postorder)."""

    handle: int
    n: int
    kop: np.ndarray       # K lower pattern, original numbering (CSC)
    koi: np.ndarray
    perm: np.ndarray      # final new -> old
    parent: np.ndarray    # etree in final numbering
    colcount: np.ndarray  # including the diagonal
    lp: np.ndarray        # column structures of L (strictly below the diagonal)
    li: np.ndarray
    super: np.ndarray     # nsuper+1 first columns
    sparent: np.ndarray
    slevel: np.ndarray
    srp: np.ndarray       # supernode row structures
    sri: np.ndarray
    nnz_l: int
    flops: float

    @property
    def nsuper(self) -> int:
        return len(self.super) - 1

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.orc_sym_free(C.c_void_p(self.handle))
            self.handle = 0


def analyze(n, m, jp, ji, perm=None, wp=None, wi=None) -> OracleSymbolic:
    """Symbolic analysis of K = W + J^T J + I with the given ordering (new->old)."""
    lib = _load()
    jp = _c(jp, np.int64)
    ji = _c(ji, np.int32)
    wp = _c(wp, np.int64)
    wi = _c(wi, np.int32)
    perm = _c(perm, np.int32)
    h = lib.orc_analyze(n, m, _p(jp), _p(ji), _p(wp), _p(wi), _p(perm))
    hv = C.c_void_p(h)
    ns = lib.orc_sym_nsuper(hv)
    nko = lib.orc_sym_nnz_korig(hv)
    nls = lib.orc_sym_nnz_lstruct(hv)
    nsr = lib.orc_sym_nnz_srows(hv)
    arrs = dict(kop=np.empty(n + 1, np.int64), koi=np.empty(nko, np.int32),
                perm=np.empty(n, np.int32), parent=np.empty(n, np.int32),
                colcount=np.empty(n, np.int32), lp=np.empty(n + 1, np.int64),
                li=np.empty(nls, np.int32), super=np.empty(ns + 1, np.int32),
                sparent=np.empty(ns, np.int32), slevel=np.empty(ns, np.int32),
                srp=np.empty(ns + 1, np.int64), sri=np.empty(nsr, np.int32))
    lib.orc_sym_export(hv, *[_p(arrs[k]) for k in ["kop", "koi", "perm", "parent", "colcount",
                                                   "lp", "li", "super", "sparent", "slevel",
                                                   "srp", "sri"]])
    return OracleSymbolic(handle=h, n=n, nnz_l=int(lib.orc_sym_nnz_l(hv)),
                          flops=float(lib.orc_sym_flops(hv)), **arrs)


def assemble(S: OracleSymbolic, m, jp, ji, jv, D, dextra=None, delta_p=0.0,
             wp=None, wi=None, wv=None) -> np.ndarray:
    """K = W + J^T diag(D) J + diag(dextra) + delta_p I on the original lower pattern."""
    lib = _load()
    kval = np.empty(len(S.koi), np.float64)
    args = [_c(jp, np.int64), _c(ji, np.int32), _c(jv, np.float64), _c(D, np.float64),
            _c(wp, np.int64), _c(wi, np.int32), _c(wv, np.float64), _c(dextra, np.float64)]
    lib.orc_assemble(C.c_void_p(S.handle), m, *[_p(a) for a in args], float(delta_p), _p(kval))
    return kval


def factor(S: OracleSymbolic, kval) -> tuple[np.ndarray, int]:
    """Left-looking Cholesky; returns (L values by column, bad) with bad = 0 or
    1 + the first column (final numbering) whose pivot is not positive."""
    lib = _load()
    kval = _c(kval, np.float64)
    lval = np.zeros(S.nnz_l, np.float64)
    bad = lib.orc_factor(C.c_void_p(S.handle), _p(kval), _p(lval))
    return lval, int(bad)


def solve(S: OracleSymbolic, lval, b) -> np.ndarray:
    lib = _load()
    b = _c(b, np.float64)
    x = np.empty(S.n, np.float64)
    lib.orc_solve(C.c_void_p(S.handle), _p(_c(lval, np.float64)), _p(b), _p(x))
    return x


def factor_ldlt(S: OracleSymbolic, kval, sign) -> tuple[np.ndarray, np.ndarray, int]:
    """Left-looking LDL^T without pivoting of a quasi-definite K; sign (original
    numbering, +1/-1) is the pivot sign each variable's block prescribes.
    Returns (unit-L values by column, d in the final numbering, bad) with bad
    = 0 or 1 + the first column whose pivot is zero or of the wrong sign."""
    lib = _load()
    kval = _c(kval, np.float64)
    sg = _c(sign, np.int8)
    lval = np.zeros(S.nnz_l, np.float64)
    dval = np.zeros(S.n, np.float64)
    bad = lib.orc_factor_ldlt(C.c_void_p(S.handle), _p(kval), _p(sg), _p(lval), _p(dval))
    return lval, dval, int(bad)


def solve_ldlt(S: OracleSymbolic, lval, dval, b) -> np.ndarray:
    lib = _load()
    x = np.empty(S.n, np.float64)
    lib.orc_solve_ldlt(C.c_void_p(S.handle), _p(_c(lval, np.float64)), _p(_c(dval, np.float64)),
                       _p(_c(b, np.float64)), _p(x))
    return x


def kmatvec(S: OracleSymbolic, kval, x) -> np.ndarray:
    lib = _load()
    y = np.empty(S.n, np.float64)
    lib.orc_kmatvec(C.c_void_p(S.handle), _p(_c(kval, np.float64)), _p(_c(x, np.float64)), _p(y))
    return y


def l_dense(S: OracleSymbolic, lval) -> np.ndarray:
    """Dense L (final numbering) from the column storage; small cases only."""
    n = S.n
    L = np.zeros((n, n))
    for j in range(n):
        base = S.lp[j] + j
        L[j, j] = lval[base]
        rows = S.li[S.lp[j]:S.lp[j + 1]]
        L[rows, j] = lval[base + 1: base + 1 + len(rows)]
    return L


def k_dense(S: OracleSymbolic, kval, final: bool = False) -> np.ndarray:
    n = S.n
    K = np.zeros((n, n))
    for j in range(n):
        for e in range(S.kop[j], S.kop[j + 1]):
            i = S.koi[e]
            K[i, j] = kval[e]
            K[j, i] = kval[e]
    if final:
        K = K[np.ix_(S.perm, S.perm)]
    return K


class _Opts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("ir_max", C.c_int32), ("tol", C.c_double),
                ("delta_p", C.c_double), ("delta_d", C.c_double), ("ir_tol", C.c_double)]


class _Res(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32),
                ("refactorizations", C.c_int32), ("objective", C.c_double),
                ("kkt", C.c_double), ("primal_res", C.c_double), ("dual_res", C.c_double),
                ("compl_res", C.c_double), ("mu", C.c_double)]


def lp_direction(S: OracleSymbolic, lp, x, s, lam, w, delta_p=1e-8, delta_d=1e-8, ir_max=3,
                 W=None):
    """Newton direction (d_x, d_s, d_lambda) of system (3) at (x, s, lambda) with
    complementarity target w, computed through the condensed system (5).
    W = (colptr, rowidx, values) of the lower triangle of the Hessian, or None."""
    lib = _load()
    mt = len(s)
    dx = np.empty(lp.n)
    ds = np.empty(mt)
    dl = np.empty(mt)
    arrs = [_c(lp.rowptr, np.int64), _c(lp.col, np.int32), _c(lp.val, np.float64),
            _c(lp.b, np.float64), _c(lp.c, np.float64), _c(lp.l, np.float64),
            _c(lp.u, np.float64), _c(x, np.float64), _c(s, np.float64), _c(lam, np.float64),
            _c(w, np.float64)]
    w3 = [None, None, None] if W is None else [_c(W[0], np.int64), _c(W[1], np.int32),
                                              _c(W[2], np.float64)]
    bad = lib.orc_lp_direction(C.c_void_p(S.handle), lp.m, *[_p(a) for a in arrs],
                               float(delta_p), float(delta_d), int(ir_max),
                               *[_p(a) for a in w3], _p(dx), _p(ds), _p(dl))
    if bad:
        raise ArithmeticError(f"non-positive pivot at column {bad - 1}")
    return dx, ds, dl


def ipm_lp(S: OracleSymbolic, lp, tol=1e-8, max_iter=500, delta_p=1e-8, delta_d=1e-8,
           ir_max=3, ir_tol=1e-12, W=None) -> dict:
    """Mehrotra predictor-corrector IPM on  min c^T x + x^T W x / 2, A x >= b,
    l <= x <= u (W = (colptr, rowidx, values) lower CSC, or None for an LP),
    solving the primal condensed system (5) at every iteration."""
    lib = _load()
    n, m = lp.n, lp.m
    mt = m + int(np.isfinite(lp.l).sum()) + int(np.isfinite(lp.u).sum())
    x = np.empty(n)
    s = np.empty(mt)
    lam = np.empty(mt)
    log_mu = np.zeros(max_iter + 1)
    log_kkt = np.zeros(max_iter + 1)
    o = _Opts(max_iter, ir_max, tol, delta_p, delta_d, ir_tol)
    r = _Res()
    arrs = [_c(lp.rowptr, np.int64), _c(lp.col, np.int32), _c(lp.val, np.float64),
            _c(lp.b, np.float64), _c(lp.c, np.float64), _c(lp.l, np.float64),
            _c(lp.u, np.float64)]
    w3 = [None, None, None] if W is None else [_c(W[0], np.int64), _c(W[1], np.int32),
                                              _c(W[2], np.float64)]
    lib.orc_ipm_lp(C.c_void_p(S.handle), m, *[_p(a) for a in arrs], *[_p(a) for a in w3],
                   C.byref(o), _p(x), _p(s), _p(lam), C.byref(r), _p(log_mu), _p(log_kkt))
    it = r.iterations
    return dict(status=r.status, iterations=it, refactorizations=r.refactorizations,
                objective=r.objective, kkt=r.kkt, primal_res=r.primal_res,
                dual_res=r.dual_res, compl_res=r.compl_res, mu=r.mu, x=x, s=s, lam=lam,
                log_mu=log_mu[:it + 1].copy(), log_kkt=log_kkt[:it + 1].copy())
