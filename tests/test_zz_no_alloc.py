"""The allocation-free solve ig_solve_csr_noalloc, called through the C ABI, against ig_solve and
against the CPU oracle.

ig_solve_csr_noalloc exists for callers that cannot allocate device memory (a fixed memory plan
or an arena owned by another framework): it keeps all of its workspace in one static device
array. This file is collected last so that a failure here comes after every other test has run;
it passes both alone in a fresh process and after the rest of the suite.

Cases: a ragged multi-tile grid and an icosphere (two calls in a row each, plus the right-hand side
given directly), k = 4 columns, and n = IG_NOALLOC_MAX_ROWS = 65536 rows (a 256 x 256 grid: the
largest tile table, start table and partial-sum block the static layout allows), each checked
element by element against the oracle's Jacobi-PCG solved to 1e-14; and faulty caller operators,
which the call reports before solving: a zero diagonal entry (IG_ERR_INVALID_ARG), a column outside
[0, n) and a row range beyond nnz (IG_ERR_INDEX_OUT_OF_RANGE), with and without info.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import assert_close, case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12105_gb300 import _native, api
    return api, _native, _native.load()


def _setup(api, V, F, t):
    dev = torch.device("cuda:0")
    n = V.shape[0]
    mesh = api.Mesh(torch.from_numpy(F).to(dev), n)
    mesh.assemble(torch.from_numpy(V).to(dev), t)
    rowptr, col = mesh.pattern()
    A, M = mesh.operator()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    return mesh, rowptr, col, A, M, stream


def _oracle_U(V, F, t, B):
    o_rowptr, o_col, o_A, _, o_M = oracle.operator(V, F, t)
    X, _, _, st = oracle.pcg_solve(o_rowptr, o_col, o_A, o_M[:, None] * B, tol=1e-14)
    assert st == oracle.OK
    return X


def _call(lib, N, rowptr, col, A, M, n, nnz, Bt, U, stream, opts, want_info=True):
    info = N.SolveInfo() if want_info else None
    st = lib.ig_solve_csr_noalloc(_p(rowptr), _p(col), _p(A), _p(M), n, nnz, _p(Bt), Bt.shape[1], _p(U), stream,
                                  ctypes.byref(opts), ctypes.byref(info) if want_info else None)
    torch.cuda.synchronize()
    return st, (info.as_dict() if want_info else None)


@pytest.mark.parametrize("name", ["grid61x53", "ico5"])
def test_noalloc_matches_solve_and_oracle_on_two_calls(env, name):
    api, N, lib = env
    V, F, t, B, T = case(name, seed=7)
    n = V.shape[0]
    mesh, rowptr, col, A, M, stream = _setup(api, V, F, t)
    Bt = torch.from_numpy(B).to("cuda:0")
    opts = api.make_opts(rel_tol=1e-12)
    U_solve = mesh.solve(Bt, opts=opts)
    U_ref = _oracle_U(V, F, t, B)
    for call in range(2):
        U = torch.full_like(Bt, float("nan"))
        st, info = _call(lib, N, rowptr, col, A, M, n, mesh.nnz, Bt, U, stream, opts)
        assert st == N.IG_OK, (call, st, info)
        assert_close(U.cpu().numpy(), U_solve.cpu().numpy(), 1e-10, f"call {call} vs ig_solve")
        assert_close(U.cpu().numpy(), U_ref, 1e-10, f"call {call} vs oracle")
        assert max(info["true_rel_residual"]) <= 1e-12 * (1 + 1e-3)
    # right-hand side given directly (M = NULL): A X = M B with M B formed by the caller
    MB = (M[:, None] * Bt).contiguous()
    U = torch.empty_like(Bt)
    st, _ = _call(lib, N, rowptr, col, A, None, n, mesh.nnz, MB, U, stream, opts, want_info=False)
    assert st == N.IG_OK
    assert_close(U.cpu().numpy(), U_ref, 1e-10, "M = NULL vs oracle")


def test_noalloc_four_columns(env):
    api, N, lib = env
    V, F, t, B, T = case("grid61x53", seed=8, k=4)
    mesh, rowptr, col, A, M, stream = _setup(api, V, F, t)
    Bt = torch.from_numpy(B).to("cuda:0")
    U = torch.full_like(Bt, float("nan"))
    st, info = _call(lib, N, rowptr, col, A, M, V.shape[0], mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-12))
    assert st == N.IG_OK and info["k"] == 4, info
    assert_close(U.cpu().numpy(), _oracle_U(V, F, t, B), 1e-10, "k = 4 vs oracle")


def test_noalloc_at_the_row_limit(env):
    """n = 65536 = IG_NOALLOC_MAX_ROWS: the static layout at its largest."""
    from paper_2602_12105_gb300 import meshgen as mg
    api, N, lib = env
    p = mg.config_grid(256, 256, seed=3)
    assert p.n == 65536
    B = np.random.default_rng(4).uniform(-1, 1, (p.n, 3))
    mesh, rowptr, col, A, M, stream = _setup(api, p.V, p.F, p.t)
    Bt = torch.from_numpy(B).to("cuda:0")
    U_ref = _oracle_U(p.V, p.F, p.t, B)
    for call in range(2):
        U = torch.full_like(Bt, float("nan"))
        st, info = _call(lib, N, rowptr, col, A, M, p.n, mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-12))
        assert st == N.IG_OK, (call, info)
        assert_close(U.cpu().numpy(), U_ref, 1e-10, f"n = 65536, call {call} vs oracle")


def test_noalloc_reports_a_zero_diagonal(env):
    """A caller operator whose row 5 has a zero diagonal entry: the set-up kernel flags it, and the
    call returns IG_ERR_INVALID_ARG, without solving, whether or not info is asked for."""
    api, N, lib = env
    V, F, t, B, T = case("grid61x53", seed=9)
    mesh, rowptr, col, A, M, stream = _setup(api, V, F, t)
    rp = rowptr.cpu().numpy()
    cl = col.cpu().numpy()
    diag = rp[5] + int(np.nonzero(cl[rp[5]:rp[6]] == 5)[0][0])
    A_bad = A.clone()
    A_bad[diag] = 0.0
    Bt = torch.from_numpy(B).to("cuda:0")
    U = torch.empty_like(Bt)
    opts = api.make_opts(rel_tol=1e-12, max_iter=40)
    st, info = _call(lib, N, rowptr, col, A_bad, M, V.shape[0], mesh.nnz, Bt, U, stream, opts)
    assert st == N.IG_ERR_INVALID_ARG and info["status"] == N.IG_ERR_INVALID_ARG, (st, info)
    st, _ = _call(lib, N, rowptr, col, A_bad, M, V.shape[0], mesh.nnz, Bt, U, stream, opts, want_info=False)
    assert st == N.IG_ERR_INVALID_ARG
    # the next call with the good operator starts clean
    st, info = _call(lib, N, rowptr, col, A, M, V.shape[0], mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-12))
    assert st == N.IG_OK, info


def test_noalloc_rejects_out_of_range_columns_before_solving(env):
    """A column index outside [0, n) in the caller's pattern is found by the set-up kernel (which
    reads every row's columns once, within the row ranges it has checked against nnz) and the call
    returns IG_ERR_INDEX_OUT_OF_RANGE without launching the solve: U keeps its contents."""
    api, N, lib = env
    V, F, t, B, T = case("grid61x53", seed=10)
    mesh, rowptr, col, A, M, stream = _setup(api, V, F, t)
    col_bad = col.clone()
    col_bad[7] = V.shape[0] + 5
    Bt = torch.from_numpy(B).to("cuda:0")
    U = torch.full_like(Bt, 3.0)
    st, info = _call(lib, N, rowptr, col_bad, A, M, V.shape[0], mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-10))
    assert st == N.IG_ERR_INDEX_OUT_OF_RANGE and info["status"] == N.IG_ERR_INDEX_OUT_OF_RANGE, (st, info)
    assert bool((U == 3.0).all())
    # a row range beyond nnz
    rp_bad = rowptr.clone()
    rp_bad[-1] = mesh.nnz + 4
    st, _ = _call(lib, N, rp_bad, col, A, M, V.shape[0], mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-10),
                  want_info=False)
    assert st == N.IG_ERR_INDEX_OUT_OF_RANGE
    st, info = _call(lib, N, rowptr, col, A, M, V.shape[0], mesh.nnz, Bt, U, stream, api.make_opts(rel_tol=1e-10))
    assert st == N.IG_OK, info


def test_noalloc_rejects_sizes_beyond_the_limit(env):
    api, N, lib = env
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    idx = torch.zeros(8, dtype=torch.int32, device="cuda:0")
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    too_many = 65536 + 1
    st = lib.ig_solve_csr_noalloc(_p(idx), _p(idx), _p(dummy), None, too_many, too_many, _p(dummy), 1, _p(out),
                                  None, None, None)
    assert st == N.IG_ERR_INVALID_ARG
    st = lib.ig_solve_csr_noalloc(_p(idx), _p(idx), _p(dummy), None, 4, 4, _p(dummy), 5, _p(out), None, None, None)
    assert st == N.IG_ERR_INVALID_ARG
