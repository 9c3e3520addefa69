"""Failure and concurrency paths of the C ABI, made on the host (no GPU fault is involved).

  * a NaN planted in M gives SFR_E_NAN (the ||M||_F pass flags it before any iteration);
  * sfr_poll with a short positive timeout on a running request gives SFR_E_TIMEOUT, and
    the request still finishes with SFR_OK;
  * a full request queue refuses sfr_submit with SFR_E_BUSY, and every accepted request
    still finishes;
  * admission under an HBM budget lets a small request run ahead of a large one that does
    not fit yet, instead of waiting behind it.
"""
import numpy as np
import pytest

from paper_1503_03004_gb300 import binding as B
from paper_1503_03004_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


class _Req:
    """Device inputs and outputs of one float64 request (kept alive until polled)."""

    def __init__(self, m, n, r, seed, **kw):
        prob = synth.planted(m, n, r, p=0.05, amp=1.0, seed=seed, dtype="f64")
        f = dict(dtype=torch.float64, device="cuda")
        self.M = torch.from_numpy(prob.M).cuda()
        self.U, self.B = torch.empty((m, r), **f), torch.empty((r, r), **f)
        self.V, self.S = torch.empty((n, r), **f), torch.empty((m, n), **f)
        self.prob = B.make_problem(m=m, n=n, r=r, M_ptr=self.M.data_ptr(), m_dtype=B.F64, rho=1.5, **kw)
        self.res = B.make_result(U_ptr=self.U.data_ptr(), B_ptr=self.B.data_ptr(), V_ptr=self.V.data_ptr(),
                                 S_ptr=self.S.data_ptr(), s_dtype=B.F64, lds=n)


def test_nan_in_m_reports_nan():
    _gpu()
    prob = synth.planted(300, 200, 5, p=0.05, amp=1.0, seed=17, dtype="f64")
    M = prob.M.copy()
    M[123, 45] = np.nan
    with B.Context(0) as ctx:
        sol = B.solve_torch(ctx, torch.from_numpy(M).cuda(), 5, rho=1.5, check=False)
        assert sol.status == B.E_NAN
        assert ctx.last_error()
        # the context stays usable
        ok = B.solve_torch(ctx, torch.from_numpy(prob.M).cuda(), 5, rho=1.5, fixed_iters=3)
        assert ok.status == B.OK


def test_poll_timeout_then_ok():
    _gpu()
    big = _Req(4096, 4096, 32, seed=5, fixed_iters=100)
    with B.Context(0, max_slots=1) as ctx:
        t = ctx.submit(big.prob, big.res)
        assert ctx.poll(t, 1000) == B.E_TIMEOUT   # 1 ms: far shorter than 100 iterations at 4096^2
        assert ctx.poll(t, -1) == B.OK
        assert big.res.iters == 100


def test_full_queue_reports_busy():
    _gpu()
    big = _Req(4096, 4096, 32, seed=6, fixed_iters=100)
    small = [_Req(64, 48, 2, seed=100 + i, fixed_iters=3) for i in range(80)]
    with B.Context(0, max_slots=1) as ctx:   # one slot: the queue holds 64 requests
        tickets = [ctx.submit(big.prob, big.res)]
        busy_at = None
        for i, q in enumerate(small):
            try:
                tickets.append(ctx.submit(q.prob, q.res))
            except B.SfrError as e:
                assert e.status == B.E_BUSY
                busy_at = i
                break
        # the slot may or may not have taken the large request off the queue yet
        assert busy_at in (63, 64), busy_at
        assert "queue full" in ctx.last_error()
        for t in tickets:
            assert ctx.poll(t, -1) == B.OK


def test_small_request_passes_a_large_one_that_does_not_fit_yet():
    _gpu()
    big1 = _Req(4096, 4096, 32, seed=7, fixed_iters=100)   # about 0.45 GB of workspace each
    big2 = _Req(4096, 4096, 32, seed=8, fixed_iters=100)
    tiny = _Req(200, 150, 4, seed=9, fixed_iters=5)
    with B.Context(0, max_slots=2, hbm_budget_bytes=700 << 20) as ctx:
        t1 = ctx.submit(big1.prob, big1.res)
        t2 = ctx.submit(big2.prob, big2.res)   # does not fit beside big1: waits for its memory
        t3 = ctx.submit(tiny.prob, tiny.res)   # fits: admitted ahead of big2
        assert ctx.poll(t3, -1) == B.OK
        assert ctx.poll(t2, 0) == B.PENDING    # big2 cannot start before big1 ends, and runs as long
        assert ctx.poll(t1, -1) == B.OK
        assert ctx.poll(t2, -1) == B.OK
