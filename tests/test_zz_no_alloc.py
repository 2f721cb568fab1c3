"""The allocation-free solve ig_solve_csr_noalloc, called through the C ABI, against ig_solve.

ig_solve_csr_noalloc exists for callers that cannot allocate device memory (a fixed memory plan
or an arena owned by another framework): it keeps all of its workspace in one static device
array. This file is collected last so that a failure here comes after every other test has run;
it passes both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import case, rel2

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


@pytest.mark.parametrize("name", ["grid61x53", "ico5"])
def test_noalloc_matches_solve_on_two_calls(env, name):
    api, N, lib = env
    V, F, t, B, T = case(name, seed=7)
    n = V.shape[0]
    dev = torch.device("cuda:0")
    mesh = api.Mesh(torch.from_numpy(F).to(dev), n)
    mesh.assemble(torch.from_numpy(V).to(dev), t)
    rowptr, col = mesh.pattern()
    A, M = mesh.operator()
    Bt = torch.from_numpy(B).to(dev)
    opts = api.make_opts(rel_tol=1e-12)
    U_ref = mesh.solve(Bt, opts=opts)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    k = Bt.shape[1]
    for call in range(2):
        U = torch.full_like(Bt, float("nan"))
        info = N.SolveInfo()
        st = lib.ig_solve_csr_noalloc(_p(rowptr), _p(col), _p(A), _p(M), n, mesh.nnz, _p(Bt), k, _p(U), stream,
                                      ctypes.byref(opts), ctypes.byref(info))
        torch.cuda.synchronize()
        assert st == N.IG_OK, (call, st, info.as_dict())
        assert rel2(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-10, call
        assert max(info.as_dict()["true_rel_residual"]) <= 1e-12 * (1 + 1e-3)
    # right-hand side given directly (M = NULL): A X = M B with M B formed by the caller
    MB = (M[:, None] * Bt).contiguous()
    U = torch.empty_like(Bt)
    st = lib.ig_solve_csr_noalloc(_p(rowptr), _p(col), _p(A), None, n, mesh.nnz, _p(MB), k, _p(U), stream,
                                  ctypes.byref(opts), None)
    torch.cuda.synchronize()
    assert st == N.IG_OK
    assert rel2(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-10


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
