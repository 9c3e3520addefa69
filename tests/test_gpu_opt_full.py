"""GPU parity of FixedRankOptFull (Algorithm 4) through the C ABI against the float64 oracle.

The oracle iterates Algorithm 3 on a fixed M literally (oracle.fradm.fixed_rank_opt_full); the
GPU runs the same iteration with both thin products reading M (P = M V on the sweep's tile
partition, W = M^T U).  Bars as for FR-ADM: 1e-9 relative on L = U B V^T for the float64 path,
1e-5 for the mixed path.  Theorem 2 gives a second, oracle-free check: the iterates converge to
the rank-r truncated SVD of M.
"""
import numpy as np
import pytest

from oracle import fradm as O
from paper_1503_03004_gb300 import binding as B
from paper_1503_03004_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-9
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _dev(prob):
    if prob.dtype == "bf16":
        return torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(prob.M).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _L(U, Bm, V):
    return U @ Bm @ V.T


def _np(sol):
    return sol.U.cpu().numpy(), sol.B.cpu().numpy(), sol.V.cpu().numpy()


def _oracle(M, r, K, V0=None, B0=None):
    m, n = M.shape
    V0 = np.eye(n, r) if V0 is None else V0
    B0 = np.eye(r) if B0 is None else B0
    return O.fixed_rank_opt_full(M, None, B0, V0, K)[-1]


def _gapped(m, n, r, seed, gap=8.0):
    """M = Q1 diag(sigma) Q2^T with sigma_1..r in [gap, 2 gap] and the rest in [0, 1]."""
    g = synth.rng(seed)
    k = min(m, n)
    Q1, _ = np.linalg.qr(g.standard_normal((m, k)))
    Q2, _ = np.linalg.qr(g.standard_normal((n, k)))
    sig = np.concatenate([np.sort(g.uniform(gap, 2 * gap, r))[::-1], np.sort(g.uniform(0.0, 1.0, k - r))[::-1]])
    return (Q1 * sig) @ Q2.T


@pytest.mark.parametrize("m,n,r,K,dtype", [
    (77, 53, 3, 1, "f64"),      # one step (Algorithm 3 once)
    (300, 200, 7, 12, "f64"),   # several 64-row / 32-column tiles, ragged tails
    (517, 1030, 25, 6, "f32"),  # m < n, float32 storage in the float64 path
    (1000, 776, 64, 5, "bf16"),  # the widest rank the library supports
])
def test_fp64_path_matches_oracle(ctx, m, n, r, K, dtype):
    prob = synth.planted(m, n, r, p=0.05, amp=10.0, seed=310 + m, dtype=dtype)
    M = prob.values_f64()
    Ur, Br, Vr = _oracle(M, r, K)
    sol = B.opt_full_torch(ctx, _dev(prob), r, tol=0.0, max_iter=K, precision=B.PREC_FP64)
    U, Bm, V = _np(sol)
    assert sol.status == B.OK and sol.iters == K
    assert _rel(_L(U, Bm, V), _L(Ur, Br, Vr)) <= FP64_TOL
    # U, B, V themselves are determined by the iteration (polar form, no gauge freedom)
    assert _rel(U, Ur) <= 1e-8 and _rel(V, Vr) <= 1e-8 and _rel(Bm, Br) <= 1e-9
    assert abs(sol.rel_change - np.linalg.norm(Br - _oracle(M, r, K - 1)[1] if K > 1 else Br - np.eye(r))
               / np.linalg.norm(Br)) <= 1e-9 + 1e-6 * sol.rel_change


@pytest.mark.parametrize("m,n,r,K,dtype", [
    (300, 200, 7, 8, "f32"),     # SIMT float32 passes
    (1000, 776, 64, 6, "bf16"),  # tensor-core passes (bfloat16 M, r > 32), ragged row and column tiles
    (2048, 1536, 40, 6, "bf16"),  # tensor-core passes, several row blocks per CTA range
])
def test_mixed_path_matches_oracle(ctx, m, n, r, K, dtype):
    prob = synth.planted(m, n, r, p=0.05, amp=10.0, seed=410 + m, dtype=dtype)
    M = prob.values_f64()
    Ur, Br, Vr = _oracle(M, r, K)
    sol = B.opt_full_torch(ctx, _dev(prob), r, tol=0.0, max_iter=K, precision=B.PREC_MIXED)
    U, Bm, V = _np(sol)
    assert sol.status == B.OK and sol.iters == K
    assert _rel(_L(U, Bm, V), _L(Ur, Br, Vr)) <= MIXED_TOL
    assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-5 and np.abs(V.T @ V - np.eye(r)).max() <= 1e-5


@pytest.mark.parametrize("precision,dtype,r", [(B.PREC_FP64, "f64", 9), (B.PREC_MIXED, "bf16", 48)])
def test_given_V0_B0_matches_oracle(ctx, precision, dtype, r):
    # Algorithm 4 from an arbitrary Stiefel V_0 and a symmetric invertible B_0 that need not be
    # SPD (Lemma 1 needs only rank(B_0) = r)
    m, n, K = 640, 384, 5
    prob = synth.planted(m, n, r, p=0.05, amp=10.0, seed=510 + r, dtype=dtype)
    M = prob.values_f64()
    g = synth.rng(77 + r)
    V0, _ = np.linalg.qr(g.standard_normal((n, r)))
    G = g.standard_normal((r, r))
    B0 = G + G.T + 2.0 * np.eye(r)
    Ur, Br, Vr = _oracle(M, r, K, V0=V0, B0=B0)
    sol = B.opt_full_torch(ctx, _dev(prob), r, V0=torch.from_numpy(V0).cuda(), B0=torch.from_numpy(B0).cuda(),
                           tol=0.0, max_iter=K, precision=precision)
    U, Bm, V = _np(sol)
    assert sol.status == B.OK
    tol = FP64_TOL if precision == B.PREC_FP64 else MIXED_TOL
    assert _rel(_L(U, Bm, V), _L(Ur, Br, Vr)) <= tol


def test_converges_to_the_truncated_svd(ctx):
    # Theorem 2: L_i = U_i B_i V_i^T -> TSVD_r(M), subspace error shrinking like (s_{r+1}/s_r)^{2i};
    # checked against numpy's SVD, independently of the oracle
    m, n, r = 600, 450, 12
    M = _gapped(m, n, r, seed=99)
    Q, s, Wt = np.linalg.svd(M, full_matrices=False)
    T = (Q[:, :r] * s[:r]) @ Wt[:r]
    # (s_{r+1}/s_r)^2 <= 1/64 here, so 20 iterations reach the float64 floor
    sol = B.opt_full_torch(ctx, torch.from_numpy(M).cuda(), r, tol=0.0, max_iter=20, precision=B.PREC_FP64)
    U, Bm, V = _np(sol)
    assert sol.status == B.OK and sol.iters == 20 and sol.rel_change <= 1e-12
    assert _rel(_L(U, Bm, V), T) <= 1e-11
    # at the fixed point B is SPD with the top r singular values as eigenvalues (Lemma 2)
    assert np.allclose(np.sort(np.linalg.eigvalsh(Bm))[::-1], s[:r], rtol=1e-10)
    assert abs(sol.lambda_min_B - s[r - 1]) <= 1e-10 * s[0]
    assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-12


def test_subspace_error_rate(ctx):
    # the per-iteration contraction of Theorem 2: ||P_{U_i} - P_{U*}|| falls by about
    # (s_{r+1}/s_r)^2 per iteration (orthogonal iteration on M M^T)
    m, n, r = 400, 300, 5
    M = _gapped(m, n, r, seed=5, gap=3.0)
    Q, s, _ = np.linalg.svd(M, full_matrices=False)
    Pstar = Q[:, :r] @ Q[:, :r].T
    errs = []
    for K in (2, 3, 4, 5, 6):
        sol = B.opt_full_torch(ctx, torch.from_numpy(M).cuda(), r, tol=0.0, max_iter=K, precision=B.PREC_FP64)
        U = sol.U.cpu().numpy()
        errs.append(np.linalg.norm(U @ U.T - Pstar, 2))
    rate = (s[r] / s[r - 1]) ** 2
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    # the error mixes components decaying like (s_{r+j}/s_r)^{2i}, j >= 1: ratios at most about
    # `rate`, and not far below it while the j = 1 component dominates
    assert np.all(ratios <= 1.1 * rate) and np.all(ratios >= 0.1 * rate), (ratios, rate)


def test_tolerance_and_iteration_cap(ctx):
    prob = synth.planted(500, 400, 10, p=0.05, amp=10.0, seed=611, dtype="f64")
    Md = _dev(prob)
    sol = B.opt_full_torch(ctx, Md, 10, tol=1e-10, max_iter=100, precision=B.PREC_FP64)
    assert sol.status == B.OK and sol.rel_change <= 1e-10 and 1 < sol.iters < 100
    capped = B.opt_full_torch(ctx, Md, 10, tol=1e-30, max_iter=3, precision=B.PREC_FP64, check=False)
    assert capped.status == B.E_NOCONV and capped.iters == 3
    # the factors of a capped run are still returned: they equal a fixed three-iteration run
    fixed = B.opt_full_torch(ctx, Md, 10, tol=0.0, max_iter=3, precision=B.PREC_FP64)
    assert torch.equal(capped.U, fixed.U) and torch.equal(capped.B, fixed.B)


def test_rank_deficient_input_is_reported(ctx):
    # rank(M) = 3 < r = 5: the Gram of M V B is singular, which Eq. 9 excludes
    g = synth.rng(3)
    M = g.standard_normal((200, 3)) @ g.standard_normal((3, 150))
    sol = B.opt_full_torch(ctx, torch.from_numpy(M).cuda(), 5, tol=0.0, max_iter=4, precision=B.PREC_FP64,
                           check=False)
    assert sol.status == B.E_RANK
    assert "rank" in ctx.last_error()


def test_host_buffers_match_device_buffers(ctx):
    prob = synth.planted(333, 222, 6, p=0.05, amp=10.0, seed=711, dtype="f32")
    dev = B.opt_full_torch(ctx, _dev(prob), 6, tol=0.0, max_iter=7, precision=B.PREC_MIXED)
    m, n, r = 333, 222, 6
    U = np.zeros((m, r))
    Bm = np.zeros((r, r))
    V = np.zeros((n, r))
    Mh = np.ascontiguousarray(prob.M)
    p = B.OptFullProblem(m=m, n=n, ldm=n, r=r, m_dtype=B.F32, M=Mh.ctypes.data, V0=None, B0=None, tol=0.0,
                         max_iter=7, precision=B.PREC_MIXED, mem=B.MEM_HOST)
    res = B.OptFullResult(U=U.ctypes.data, B=Bm.ctypes.data, V=V.ctypes.data, iters=0, rel_change=0.0,
                          lambda_min_B=0.0, status=B.PENDING)
    assert ctx.opt_full(p, res) == B.OK and res.iters == 7
    assert np.array_equal(U, dev.U.cpu().numpy()) and np.array_equal(V, dev.V.cpu().numpy())
    assert np.array_equal(Bm, dev.B.cpu().numpy())


def test_invalid_arguments_are_refused(ctx):
    M = torch.zeros((10, 8), dtype=torch.float64, device="cuda")
    p = B.OptFullProblem(m=10, n=8, ldm=8, r=9, m_dtype=B.F64, M=M.data_ptr(), V0=None, B0=None, tol=0.0, max_iter=3,
                         precision=B.PREC_FP64, mem=B.MEM_DEVICE)
    res = B.OptFullResult()
    assert ctx.opt_full(p, res) == B.E_INVAL and res.status == B.E_INVAL
    p.r, p.max_iter = 4, 0
    assert ctx.opt_full(p, res) == B.E_INVAL
    p.max_iter, p.M = 3, None
    assert ctx.opt_full(p, res) == B.E_INVAL
    # a nonsymmetric B_0 (the projector's (B G B)^{-1/2} needs B = B^T)
    B0 = torch.eye(4, dtype=torch.float64, device="cuda")
    B0[0, 1] = 0.5
    p.M, p.B0 = M.data_ptr(), B0.data_ptr()
    assert ctx.opt_full(p, res) == B.E_INVAL and "symmetric" in ctx.last_error()


def test_square16384_r64_bf16_full_size(ctx):
    # the benchmark workload's matrix through the tensor-core passes, as bench.py --opt-full times
    # it; at this size the checks are properties that hold at any size: orthonormal factors,
    # symmetric B, and the fixed-point equations M V = U B and M^T U = V B of the truncated SVD
    # (Theorem 2), evaluated here with float64 products of the stored bfloat16 M
    prob = synth.square_large(16384, 64, dtype="bf16", seed=1001)
    Md = _dev(prob)
    sol = B.opt_full_torch(ctx, Md, 64, tol=1e-6, max_iter=30, precision=B.PREC_MIXED)
    assert sol.status == B.OK and sol.rel_change <= 1e-6
    r = 64
    eye = torch.eye(r, dtype=torch.float64, device="cuda")
    assert float((sol.U.T @ sol.U - eye).abs().max()) <= 1e-5
    assert float((sol.V.T @ sol.V - eye).abs().max()) <= 1e-5
    assert float((sol.B - sol.B.T).abs().max()) <= 1e-12 * float(sol.B.abs().max())
    nb = float(torch.linalg.norm(sol.B))
    MV = torch.empty((16384, r), dtype=torch.float64, device="cuda")
    MtU = torch.zeros((16384, r), dtype=torch.float64, device="cuda")
    for i0 in range(0, 16384, 2048):
        blk = Md[i0:i0 + 2048].double()
        MV[i0:i0 + 2048] = blk @ sol.V
        MtU += blk.T @ sol.U[i0:i0 + 2048]
    assert float(torch.linalg.norm(MV - sol.U @ sol.B)) <= 1e-5 * nb
    assert float(torch.linalg.norm(MtU - sol.V @ sol.B)) <= 1e-5 * nb
    assert sol.lambda_min_B > 0
