"""Serving: sfr_submit / sfr_poll with several slots (continuous batching of independent solves).

Requests of uneven shape and precision run concurrently on the device, each slot on its own
stream; every result must equal the same problem solved alone with sfr_solve (the kernels are
deterministic, so equality is exact), and the HBM budget must gate admission.
"""
import numpy as np
import pytest

from paper_1503_03004_gb300 import binding as B
from paper_1503_03004_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(prob):
    if prob.dtype == "bf16":
        return torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(prob.M).cuda()


def _request(prob, precision, **kw):
    m, n = prob.shape
    r = prob.r
    Md = _dev(prob)
    f64 = dict(dtype=torch.float64, device="cuda")
    U, Bm, V = torch.empty((m, r), **f64), torch.empty((r, r), **f64), torch.empty((n, r), **f64)
    S = torch.empty((m, n), dtype=torch.float32, device="cuda")
    code = {"f64": B.F64, "f32": B.F32, "bf16": B.BF16}[prob.dtype]
    p = B.make_problem(m=m, n=n, r=r, M_ptr=Md.data_ptr(), m_dtype=code, precision=precision, **kw)
    res = B.make_result(U_ptr=U.data_ptr(), B_ptr=Bm.data_ptr(), V_ptr=V.data_ptr(), S_ptr=S.data_ptr(),
                        s_dtype=B.F32, lds=n)
    return dict(M=Md, U=U, B=Bm, V=V, S=S, p=p, res=res)


def _workload():
    out = []
    for i, (m, n, r, dt, prec) in enumerate([(300, 200, 5, "f64", B.PREC_FP64), (700, 96, 3, "f32", B.PREC_MIXED),
                                             (512, 512, 40, "bf16", B.PREC_MIXED), (256, 384, 10, "f64", B.PREC_FP64),
                                             (1024, 64, 8, "bf16", B.PREC_MIXED), (640, 640, 64, "bf16", B.PREC_MIXED),
                                             (128, 1000, 4, "f32", B.PREC_FP64), (900, 300, 25, "bf16", B.PREC_MIXED)]):
        prob = synth.planted(m, n, r, p=0.06, amp=50.0, seed=500 + i, dtype=dt)
        out.append((prob, prec))
    return out


def test_concurrent_requests_equal_solo_solves():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    kw = dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    work = _workload()
    with B.Context(0, max_slots=4) as ctx:
        solo = []
        for prob, prec in work:
            q = _request(prob, prec, **kw)
            assert ctx.solve(q["p"], q["res"]) == B.OK, ctx.last_error()
            solo.append(q)
        mixed = [_request(prob, prec, **kw) for prob, prec in work]
        tickets = [ctx.submit(q["p"], q["res"]) for q in mixed]
        for t in tickets:
            assert ctx.poll(t, -1) == B.OK, ctx.last_error()
    for a, b in zip(solo, mixed):
        assert a["res"].iters == b["res"].iters
        for key in ("U", "B", "V", "S"):
            assert torch.equal(a[key], b[key]), key


def test_poll_reports_pending_then_done():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    prob = synth.planted(2048, 2048, 64, p=0.05, amp=50.0, seed=77, dtype="bf16")
    with B.Context(0, max_slots=2) as ctx:
        q = _request(prob, B.PREC_MIXED, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
        t = ctx.submit(q["p"], q["res"])
        first = ctx.poll(t, 0)
        assert first in (B.PENDING, B.OK)
        assert ctx.poll(t, -1) == B.OK
        assert q["res"].status == B.OK


def test_hbm_budget_gates_admission():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    small = synth.planted(200, 150, 4, p=0.05, amp=1.0, seed=3, dtype="f64")
    big = synth.planted(3000, 3000, 16, p=0.05, amp=1.0, seed=4, dtype="f64")
    with B.Context(0, max_slots=3, hbm_budget_bytes=64 << 20) as ctx:
        qs = [_request(small, B.PREC_FP64, fixed_iters=5), _request(big, B.PREC_FP64, fixed_iters=5),
              _request(small, B.PREC_FP64, fixed_iters=5)]
        ts = [ctx.submit(q["p"], q["res"]) for q in qs]
        st = [ctx.poll(t, -1) for t in ts]
    assert st == [B.OK, B.E_NOMEM, B.OK]
    assert torch.equal(qs[0]["U"], qs[2]["U"])


def _batch_workload():
    # the serving-stream shapes: uneven m, n, r in {3, 5, 10, 25}, bf16 and f32 storage, rows with
    # and without 16-byte alignment (n % 4), tall-skinny ones with many W-pass row chunks
    out = []
    shapes = [(300, 40, 3), (2100, 133, 10), (777, 512, 25), (4096, 17, 5), (256, 256, 25), (1500, 96, 10),
              (8192, 48, 3), (650, 301, 5), (3000, 200, 25), (999, 64, 10), (5000, 510, 5), (400, 130, 25)]
    for i, (m, n, r) in enumerate(shapes):
        dt = "f32" if i % 3 == 2 else "bf16"
        out.append(synth.planted(m, n, r, p=0.02 + 0.01 * (i % 10), amp=50.0, seed=900 + i, dtype=dt))
    return out


def test_grouped_engine_equals_solo_solves():
    # every request of the batch runs exactly the kernels sfr_solve runs for it (grouped launches
    # with each problem's own grid and arguments): the results must be identical, bit for bit,
    # whatever else is in the batch; an ineligible request (r = 40, tensor cores) goes to a slot
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    kw = dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    work = [(p, B.PREC_MIXED) for p in _batch_workload()]
    work.append((synth.planted(512, 512, 40, p=0.05, amp=50.0, seed=990, dtype="bf16"), B.PREC_MIXED))
    with B.Context(0) as ctx:
        solo = []
        for prob, prec in work:
            q = _request(prob, prec, **kw)
            assert ctx.solve(q["p"], q["res"]) == B.OK, ctx.last_error()
            solo.append(q)
    for cap in (3, 16):  # batches smaller than the stream (admission as slots free) and larger
        with B.Context(0, max_batch=cap, max_slots=2) as ctx:
            mixed = [_request(prob, prec, **kw) for prob, prec in work]
            tickets = [ctx.submit(q["p"], q["res"]) for q in mixed]
            for t in tickets:
                assert ctx.poll(t, -1) == B.OK, ctx.last_error()
        for a, q in zip(solo, mixed):
            assert q["res"].iters == a["res"].iters
            assert q["res"].rel_residual == a["res"].rel_residual
            for k in ("U", "B", "V", "S"):
                assert torch.equal(q[k], a[k]), k
            assert q["res"].lambda_min_B == a["res"].lambda_min_B


def test_grouped_engine_reports_each_outcome():
    # a request whose first thin product P_1 = M[:, :r] has a zero column fails alone with
    # SFR_E_RANK (the r x r Gram has an exact zero eigenvalue), one with a NaN in M with
    # SFR_E_NAN, a capped one with SFR_E_NOCONV after exactly max_iter iterations, a
    # fixed-iteration one runs exactly its count; every outcome equals the solo solve's, and the
    # requests sharing the batch are unaffected
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    work = _batch_workload()
    Mr = work[2].M.copy()            # float32 storage
    Mr[:, 2] = 0.0
    rankdef = (synth.Problem(M=Mr, dtype="f32", r=4), dict(rho=1.5, mu0=0.05, fixed_iters=3))
    Mn = work[5].M.copy() if work[5].dtype == "f32" else work[8].M.copy()
    Mn[17, 11] = np.nan
    nan = (synth.Problem(M=Mn, dtype="f32", r=5), dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300))
    good = [(p, dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)) for p in work[:4]]
    capped = (work[5], dict(rho=1.5, mu0=0.05, tol=1e-14, max_iter=7))
    fixed = (work[6], dict(rho=1.5, mu0=0.05, fixed_iters=5))
    reqs = [rankdef, nan] + good + [capped, fixed]
    with B.Context(0) as ctx:
        solo = []
        for prob, kw in reqs:
            q = _request(prob, B.PREC_MIXED, **kw)
            ctx.solve(q["p"], q["res"])
            solo.append(q)
    with B.Context(0, max_batch=8) as ctx:
        qs = [_request(prob, B.PREC_MIXED, **kw) for prob, kw in reqs]
        tickets = [ctx.submit(q["p"], q["res"]) for q in qs]
        status = [ctx.poll(t, -1) for t in tickets]
    assert status == [q["res"].status for q in solo]
    assert status[0] == B.E_RANK and status[1] == B.E_NAN
    assert all(s == B.OK for s in status[2:6])
    assert status[6] == B.E_NOCONV and qs[6]["res"].iters == 7
    assert status[7] == B.OK and qs[7]["res"].iters == 5
    for a, q in zip(solo[2:], qs[2:]):
        assert q["res"].iters == a["res"].iters
        for k in ("U", "B", "V", "S"):
            assert torch.equal(q[k], a[k]), k
