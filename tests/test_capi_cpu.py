"""The C-ABI library loads, exports every declared entry point, and its host
symbolic analysis matches the oracle bit for bit. CPU only (no compute call
touches a GPU: ipm_create and kkt_analyze are host-only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import gen
import oracle
import paper_2508_16094_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return gb.load()


def _declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^IPM_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(gb.EXPORTED) <= set(names)


def _cases():
    yield "grid5", gen.grid_lp(5, seed=2), gen.nd_order_grid3d(5, leaf=16)
    yield "grid6x4x3", gen.grid_lp(6, 4, 3, seed=3), gen.nd_order_grid3d(6, 4, 3, leaf=8)
    yield "grid9", gen.grid_lp(9, seed=4), gen.nd_order_grid3d(9)
    lp = gen.random_lp(300, 150, 5, seed=5)
    yield "random300_md", lp, gen.lp_ordering(lp)
    lp = gen.random_lp(120, 200, 3, seed=6)
    yield "random120_id", lp, None


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_symbolic_bit_exact_vs_oracle(lib, case):
    _, lp, perm = case
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
    info = ctx.kkt_analyze(perm)
    got = ctx.kkt_symbolic_export()
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    for k in ["perm", "parent", "colcount", "super", "sparent", "slevel", "srp", "sri"]:
        np.testing.assert_array_equal(got[k], getattr(S, k), err_msg=k)
    assert info.nnz_l == S.nnz_l
    assert info.flops == S.flops
    assert info.nsuper == S.nsuper
    assert info.nnz_k == len(S.koi)
    assert info.m_tot == lp.m + 2 * lp.n
    ctx.close()


def test_symbolic_special_patterns(lib):
    n = 9
    # diagonal only
    ctx = gb.IpmContext(n, 0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    info = ctx.kkt_analyze()
    assert info.nnz_l == n and info.nsuper >= 1
    # dense row: one supernode of n columns
    ctx = gb.IpmContext(n, 1, np.array([0, n], np.int64), np.arange(n, dtype=np.int32))
    info = ctx.kkt_analyze()
    assert info.nsuper == 1 and info.nnz_l == n * (n + 1) // 2 and info.max_ncol == n


def test_argument_errors(lib):
    lp = gen.grid_lp(3, seed=1)
    # unsorted row
    col = lp.col.copy()
    col[0], col[1] = col[1], col[0]
    with pytest.raises(gb.IpmError) as e:
        gb.IpmContext(lp.n, lp.m, lp.rowptr, col)
    assert e.value.status == 1
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
    with pytest.raises(gb.IpmError) as e:
        ctx.kkt_analyze(np.zeros(lp.n, np.int32))  # not a permutation
    assert e.value.status == 1
    # out-of-order: factor before anything
    st, _ = ctx.kkt_factor(gb.IPM_FP64, raise_on_error=False)
    assert st == 2
    # workspace size is reported and covers the FP64 factor
    info = ctx.kkt_analyze(None)
    assert info.workspace_bytes >= 8 * info.factor_entries


def test_options_cannot_enable_learned_after_analysis():
    lp = gen.grid_lp(6, seed=24)
    o = gb.default_options(precision=4, storage_fp64=0)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    ctx.kkt_analyze(gen.nd_order_grid3d(6))
    with pytest.raises(gb.IpmError):
        ctx.ipm_set_options(learned=1)


def test_grid_nlp_pattern_matches_generator():
    """The library's grid-NLP patterns and bounds are the generator's (the
    oracle evaluates on the generator's)."""
    for N, vb in ((5, 1), (12, 1), (7, 0)):
        pt = gb.ipm_grid_nlp_pattern(N, v_bounded=vb)
        P = gen.grid_nlp(N, v_bounded=vb)
        assert pt["n"] == P.n and pt["m"] == P.m
        for a, b in (("rowptr", P.rowptr), ("col", P.col), ("wp", P.wp), ("wi", P.wi),
                     ("l", P.l), ("u", P.u)):
            assert np.array_equal(pt[a], b), a
    with pytest.raises(gb.IpmError):
        gb.ipm_grid_nlp_pattern(1)


@pytest.mark.parametrize("form", ["dual", "augmented"])
@pytest.mark.parametrize("case", ["grid5", "random120"])
def test_formulation_symbolic_bit_exact_vs_oracle(lib, form, case):
    """The systems of the dual condensed (6) and augmented (4) formulations:
    the library builds their pattern and analyses it like the oracle does the
    pattern it builds on its own (oracle/forms.py)."""
    from oracle import forms
    if case == "grid5":
        lp = gen.grid_lp(5, seed=2)
        nd = gen.nd_order_grid3d(5, leaf=16)
        perm = nd if form == "dual" else np.concatenate([[p, lp.n + p] for p in nd]).astype(np.int32)
    else:
        lp = gen.random_lp(120, 80, 3, seed=6)
        perm = None
    o = gb.default_options(formulation=gb.IPM_FORM_DUAL if form == "dual" else gb.IPM_FORM_AUGMENTED)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    info = ctx.kkt_analyze(perm)
    got = ctx.kkt_symbolic_export()
    mt = lp.m + 2 * lp.n
    one = np.ones(mt)
    if form == "dual":
        S, _, _ = forms.dual_system(lp, one, one, np.ones(lp.n), 1e-8, 1e-8, perm)
        assert info.n == lp.m and ctx.kkt_order() == lp.m
    else:
        S, _, _ = forms.augmented_system(lp, one, one, np.ones(lp.n), 1e-8, 1e-8, perm)
        assert info.n == lp.n + lp.m and ctx.kkt_order() == lp.n + lp.m
    for k in ["perm", "parent", "colcount", "super", "sparent", "slevel", "srp", "sri"]:
        np.testing.assert_array_equal(got[k], getattr(S, k), err_msg=k)
    assert info.nnz_l == S.nnz_l and info.m_tot == mt


def test_dual_formulation_rejects_a_full_hessian(lib):
    n = 4
    rp = np.array([0, 2, 4], np.int64)
    cl = np.array([0, 1, 2, 3], np.int32)
    wp = np.array([0, 2, 3, 4, 5], np.int64)  # W has the off-diagonal entry (1, 0)
    wi = np.array([0, 1, 1, 2, 3], np.int32)
    o = gb.default_options(formulation=gb.IPM_FORM_DUAL)
    ctx = gb.IpmContext(n, 2, rp, cl, None, None, wp, wi, options=o)
    with pytest.raises(gb.IpmError) as e:
        ctx.kkt_analyze(None)
    assert e.value.status == 10  # IPM_ERR_UNSUPPORTED


def test_create_pattern_matches_create():
    """ipm_create_pattern (the pattern as one struct) builds the same context
    as ipm_create: identical symbolic analysis, and a NULL pattern is refused."""
    lp = gen.grid_lp(6, 5, 4, seed=7)
    perm = np.ascontiguousarray(gen.nd_order_grid3d(6, 5, 4), dtype=np.int32)
    h, keep = gb.ipm_create_pattern(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
    lib = gb.load()
    try:
        info = gb.SymbolicInfo()
        assert lib.kkt_analyze(h, perm.ctypes.data_as(C.c_void_p), C.byref(info)) == 0
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
        ref = ctx.kkt_analyze(perm)
        for f in ("n", "nnz_l", "nsuper", "nlevels", "flops", "workspace_bytes"):
            assert getattr(info, f) == getattr(ref, f), f
    finally:
        lib.ipm_destroy(h)
    out = C.c_void_p()
    o = gb.default_options()
    assert lib.ipm_create_pattern(4, 4, None, C.byref(o), None, C.byref(out)) == 1


def test_fp64_tc_sizes_slice_storage(lib):
    """options.fp64_tc makes kkt_analyze size FP64 storage plus the BF16 slice
    planes (7 x 2 bytes per factor entry, rows padded to 8) and their exponents."""
    lp = gen.grid_lp(9, seed=3)
    perm = gen.nd_order_grid3d(9)
    ws = []
    for tc in (0, 1):
        o = gb.default_options(storage_fp64=1, fp64_tc=tc)
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
        info = ctx.kkt_analyze(perm)
        ws.append(info.workspace_bytes)
    extra = (ws[1] - ws[0]) / info.factor_entries
    assert 14.0 <= extra <= 15.0, extra
