"""sfr_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (processes whose device memory belongs to a fixed pool or a
framework allocator, paths that may not take the allocator's locks) get all
workspace from a fixed __device__ array inside the library.  This checks,
through the C ABI, that two calls in a row give the same factors and S as
sfr_solve within the parity tolerance of each precision path (float64: 1e-9,
mixed: 1e-5), and that an oversized problem is refused.  The file is named to
be collected last.
"""
import numpy as np
import pytest

from paper_1503_03004_gb300 import binding as B
from paper_1503_03004_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-9


def _buffers(m, n, r):
    f = dict(dtype=torch.float64, device="cuda")
    return (torch.empty((m, r), **f), torch.empty((r, r), **f), torch.empty((n, r), **f), torch.empty((m, n), **f))


def _run(call, Md, m, n, r, m_dtype=B.F64, **kw):
    U, Bm, V, S = _buffers(m, n, r)
    p = B.make_problem(m=m, n=n, r=r, M_ptr=Md.data_ptr(), m_dtype=m_dtype, **kw)
    res = B.make_result(U_ptr=U.data_ptr(), B_ptr=Bm.data_ptr(), V_ptr=V.data_ptr(), S_ptr=S.data_ptr(),
                        s_dtype=B.F64, lds=n)
    st = call(p, res)
    return st, res, U, Bm, V, S


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("kw", [dict(fixed_iters=7), dict(mu0=0.05, tol=1e-9)])
def test_noalloc_matches_solve_twice(kw):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m, n, r = 500, 500, 25
    prob = synth.square_fp64_500()
    Md = torch.from_numpy(prob.M).cuda()
    with B.Context(0) as ctx:
        st, ref, U0, B0, V0, S0 = _run(ctx.solve, Md, m, n, r, **kw)
        assert st == B.OK, ctx.last_error()
        L0 = U0 @ B0 @ V0.T
        for _ in range(2):
            st, res, U, Bm, V, S = _run(ctx.solve_noalloc, Md, m, n, r, **kw)
            assert st == B.OK, ctx.last_error()
            assert res.iters == ref.iters
            assert _rel(U @ Bm @ V.T, L0) <= TOL
            assert _rel(S, S0) <= 1e-8
            assert abs(res.rel_residual - ref.rel_residual) <= 1e-6 * max(ref.rel_residual, 1e-300)


@pytest.mark.parametrize("m,n,r", [(500, 500, 25), (384, 640, 64)])
def test_noalloc_mixed_matches_solve_twice(m, n, r):
    # mixed path with bfloat16 M: the no-alloc call runs the SIMT passes (also at r = 64, where
    # sfr_solve takes the tensor-core kernels); both must reach tol and agree to the mixed bar
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    prob = synth.planted(m, n, r, p=0.05, amp=50.0, seed=m + n + r, dtype="bf16")
    Md = torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    kw = dict(m_dtype=B.BF16, mu0=0.05, rho=1.5, tol=1e-9, max_iter=300, precision=B.PREC_MIXED)
    with B.Context(0) as ctx:
        st, ref, U0, B0, V0, S0 = _run(ctx.solve, Md, m, n, r, **kw)
        assert st == B.OK, ctx.last_error()
        L0 = U0 @ B0 @ V0.T
        for _ in range(2):
            st, res, U, Bm, V, S = _run(ctx.solve_noalloc, Md, m, n, r, **kw)
            assert st == B.OK, ctx.last_error()
            assert res.path == 0 and res.rel_residual <= 1e-9
            assert _rel(U @ Bm @ V.T, L0) <= 1e-5
            assert _rel(S, S0) <= 1e-4


def test_noalloc_refuses_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m, n, r = 4096, 4096, 8
    Md = torch.ones((m, n), dtype=torch.float64, device="cuda")
    with B.Context(0) as ctx:
        p = B.make_problem(m=m, n=n, r=r, M_ptr=Md.data_ptr(), m_dtype=B.F64, fixed_iters=1)
        res = B.make_result()
        assert ctx.solve_noalloc(p, res) == B.E_NOMEM
        assert "no-alloc scratch" in ctx.last_error()
