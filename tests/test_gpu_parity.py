"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (stated by the workload definitions):
  * float64 path:  ||L_gpu - L_oracle||_F / ||L_oracle||_F <= 1e-9, and the same
    support of S except entries whose |z| lies within 1e-9 (relative) of the
    threshold 1/mu (z = M - L + Y_prev/mu of the last iteration);
  * mixed path (float32 sweep):  ||L_gpu - L_oracle||_F / ||L_oracle||_F <= 1e-5.
Inputs are seeded synthetic matrices; both sides see the same stored values.
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
        t = torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(prob.M)
    return t.cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_L(sol):
    return (sol.U @ sol.B @ sol.V.T).cpu().numpy()


def _support_ok(S_gpu, ref, M):
    z = M - ref.L + ref.Y_prev / ref.mu_last
    thr = 1.0 / ref.mu_last
    near = np.abs(np.abs(z) - thr) <= 1e-9 * max(1.0, np.abs(z).max())
    diff = (S_gpu != 0) != (ref.S != 0)
    return int(np.count_nonzero(diff & ~near))


@pytest.mark.parametrize("m,n,r,K", [
    (77, 53, 3, 1),
    (77, 53, 3, 4),
    (130, 70, 8, 6),
    (200, 150, 17, 5),
    (96, 300, 1, 7),
    (300, 280, 64, 3),
    (3000, 40, 3, 6),
])
def test_fp64_fixed_iterations_match_oracle(ctx, m, n, r, K):
    prob = synth.planted(m, n, r, p=0.08, amp=1.0, seed=m * 7 + n + r, dtype="f64")
    M = prob.values_f64()
    ref = O.fr_adm(M, r, rho=1.5, fixed_iters=K)
    sol = B.solve_torch(ctx, _dev(prob), r, fixed_iters=K, rho=1.5)
    assert sol.iters == K
    assert _rel(_gpu_L(sol), ref.L) <= FP64_TOL
    np.testing.assert_allclose(sol.B.cpu().numpy(), ref.B, atol=FP64_TOL * np.abs(ref.B).max())
    assert _support_ok(sol.S.cpu().numpy(), ref, M) == 0
    # S = P_ST(M - L + Y_prev/mu) moves by no more than L does: hold it to the L bar in L's scale
    S = sol.S.cpu().numpy()
    assert np.linalg.norm(S - ref.S) <= FP64_TOL * np.linalg.norm(ref.L)


def test_fp64_500_r25_to_convergence(ctx):
    # 500 x 500, r = 25, 10% outliers in [-50, 50], float64; mu0 = 0.05, rho = 1.5, tol 1e-9
    prob = synth.square_fp64_500()
    M = prob.values_f64()
    ref = O.fr_adm(M, 25, rho=1.5, mu0=0.05, tol=1e-9)
    sol = B.solve_torch(ctx, _dev(prob), 25, rho=1.5, mu0=0.05, tol=1e-9)
    assert sol.iters == ref.iters
    assert sol.rel_residual <= 1e-9
    L = _gpu_L(sol)
    assert _rel(L, ref.L) <= FP64_TOL
    assert _support_ok(sol.S.cpu().numpy(), ref, M) == 0
    L0 = prob.U0 @ prob.V0.T
    assert _rel(L, L0) <= 1e-7            # planted recovery
    U, V = sol.U.cpu().numpy(), sol.V.cpu().numpy()
    np.testing.assert_allclose(U.T @ U, np.eye(25), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(25), atol=1e-12)
    assert sol.lambda_min_B > 0


def test_paper_table1_recipe_on_gpu(ctx):
    prob = synth.paper_table1(500, 10)
    M = prob.values_f64()
    ref = O.fr_adm(M, 10, rho=1.5, tol=1e-9)
    sol = B.solve_torch(ctx, _dev(prob), 10, rho=1.5, tol=1e-9)
    assert sol.iters == ref.iters == 28
    assert _rel(_gpu_L(sol), ref.L) <= FP64_TOL


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_mixed_matches_oracle(ctx, dtype):
    prob = synth.planted(640, 520, 10, p=0.05, amp=50.0, seed=11, dtype=dtype)
    M = prob.values_f64()
    ref = O.fr_adm(M, 10, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), 10, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300,
                        precision=B.PREC_MIXED, check=False)
    assert ref.converged
    assert sol.status == B.OK and sol.rel_residual <= 1e-9
    assert sol.path == 0                   # r = 10: the SIMT passes
    assert _rel(_gpu_L(sol), ref.L) <= MIXED_TOL


@pytest.mark.parametrize("m,n,r,dtype", [
    (517, 333, 10, "f32"),    # n % 4 != 0: the element-load variants of the float32 passes
    (301, 258, 7, "bf16"),    # the same with bfloat16 M
    (96, 3001, 5, "f32"),     # few rows, many column tiles: several splits, several tiles per split
    (2048, 1000, 20, "bf16"),  # cp.async-pipelined passes at r = 20 (padded to 32), ragged tiles
    (517, 336, 10, "f32"),    # pipelined passes with a ragged last row block (m % 64 != 0)
    (1003, 1024, 24, "bf16"),  # the same with bfloat16 M and r = 24
])
def test_mixed_simt_passes_match_oracle(ctx, m, n, r, dtype):
    prob = synth.planted(m, n, r, p=0.05, amp=50.0, seed=m * 7 + n, dtype=dtype)
    M = prob.values_f64()
    ref = O.fr_adm(M, r, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), r, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300, precision=B.PREC_MIXED,
                        s_dtype=B.F32)
    assert sol.status == B.OK and sol.rel_residual <= 1e-9
    assert _rel(_gpu_L(sol), ref.L) <= MIXED_TOL


def test_mixed_square_r64_bf16_recipe(ctx):
    # the 16384 x 16384 r = 64 recipe (5% outliers in [-50, 50], bf16 storage) at 1024 x 1024
    prob = synth.planted(1024, 1024, 64, p=0.05, amp=50.0, seed=1001, dtype="bf16")
    M = prob.values_f64()
    ref = O.fr_adm(M, 64, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), 64, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300, precision=B.PREC_MIXED,
                        s_dtype=B.F32)
    assert abs(sol.iters - ref.iters) <= 2
    assert _rel(_gpu_L(sol), ref.L) <= MIXED_TOL
    assert _rel(sol.S.cpu().numpy().astype(np.float64), ref.S) <= 1e-4


@pytest.mark.parametrize("m,n,r", [(1000, 776, 40), (384, 640, 64), (1152, 1088, 33)])
def test_tensor_core_path_matches_oracle(ctx, m, n, r):
    # bfloat16 storage with 33 <= r <= 64 takes the tcgen05 path; ragged m and n (not multiples
    # of the 128-row / 64-column tiles) exercise the TMA bounds handling.  The mixed-path bar
    # applies to the converged result (early iterates carry bfloat16 rounding of a large Delta).
    prob = synth.planted(m, n, r, p=0.05, amp=50.0, seed=m + n + r, dtype="bf16")
    M = prob.values_f64()
    ref = O.fr_adm(M, r, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), r, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300, precision=B.PREC_MIXED,
                        s_dtype=B.F32)
    assert sol.path & B.PATH_TC            # the tcgen05 sweep and W pass ran
    assert abs(sol.iters - ref.iters) <= 3
    assert _rel(_gpu_L(sol), ref.L) <= MIXED_TOL
    assert _rel(sol.S.cpu().numpy().astype(np.float64), ref.S) <= 1e-4


def test_fp64_path_with_low_precision_storage(ctx):
    prob = synth.planted(256, 192, 6, p=0.1, amp=1.0, seed=5, dtype="bf16")
    M = prob.values_f64()
    ref = O.fr_adm(M, 6, rho=1.5, fixed_iters=12)
    sol = B.solve_torch(ctx, _dev(prob), 6, rho=1.5, fixed_iters=12)
    assert _rel(_gpu_L(sol), ref.L) <= FP64_TOL


def test_host_memory_mode_matches_device_mode(ctx):
    prob = synth.planted(150, 120, 5, p=0.1, amp=1.0, seed=21, dtype="f64")
    dev = B.solve_torch(ctx, _dev(prob), 5, fixed_iters=9)
    M = np.ascontiguousarray(prob.M)
    U = np.empty((150, 5)); Bm = np.empty((5, 5)); V = np.empty((120, 5)); S = np.empty((150, 120))
    p = B.make_problem(m=150, n=120, r=5, M_ptr=M.ctypes.data, m_dtype=B.F64, fixed_iters=9, mem=B.MEM_HOST)
    res = B.make_result(U_ptr=U.ctypes.data, B_ptr=Bm.ctypes.data, V_ptr=V.ctypes.data, S_ptr=S.ctypes.data,
                        s_dtype=B.F64, lds=120)
    assert ctx.solve(p, res) == B.OK
    np.testing.assert_array_equal(U, dev.U.cpu().numpy())
    np.testing.assert_array_equal(S, dev.S.cpu().numpy())


def test_frnys_matches_oracle(ctx):
    m, n, r, l = 400, 300, 4, 40
    prob = synth.planted(m, n, r, p=0.05, amp=1.0, seed=91, dtype="f64")
    M = prob.values_f64()
    perm = synth.row_permutation(m, 92)
    ref = O.fr_nys(M, r, l, perm, rho=1.5, mu0=0.1, tol=1e-10)
    sol = B.solve_torch(ctx, _dev(prob), r, nys_l=l, nys_perm=torch.from_numpy(perm).cuda(), rho=1.5, mu0=0.1,
                        tol=1e-10, want_L=True)
    assert sol.iters == ref.left.iters + ref.top.iters
    assert _rel(sol.L.cpu().numpy(), ref.L) <= FP64_TOL
    assert _rel(sol.S.cpu().numpy(), ref.S) <= 1e-6
    # the factors: L = U B V^T with U, V orthonormal and B = diag(sigma), sigma decreasing
    U, Bm, V = (x.cpu().numpy() for x in (sol.U, sol.B, sol.V))
    assert _rel(U @ Bm @ V.T, ref.L) <= FP64_TOL
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-12)
    sig = np.diag(Bm)
    assert np.count_nonzero(Bm - np.diag(sig)) == 0 and np.all(np.diff(sig) <= 0) and sig[-1] > 0
    assert sol.lambda_min_B == pytest.approx(sig[-1])
    np.testing.assert_allclose(sig, np.linalg.svd(ref.L, compute_uv=False)[:r], rtol=1e-9)


def test_submit_poll_equals_solve(ctx):
    probs = [synth.planted(120 + 40 * i, 90 + 10 * i, 3 + i, p=0.08, amp=1.0, seed=300 + i, dtype="f64") for i in range(4)]
    alone = [B.solve_torch(ctx, _dev(p), p.r, fixed_iters=8) for p in probs]
    keep, tickets = [], []
    for p in probs:
        Md = _dev(p)
        m, n = p.shape
        U = torch.empty((m, p.r), dtype=torch.float64, device="cuda")
        Bm = torch.empty((p.r, p.r), dtype=torch.float64, device="cuda")
        V = torch.empty((n, p.r), dtype=torch.float64, device="cuda")
        S = torch.empty((m, n), dtype=torch.float64, device="cuda")
        prob = B.make_problem(m=m, n=n, r=p.r, M_ptr=Md.data_ptr(), m_dtype=B.F64, fixed_iters=8)
        res = B.make_result(U_ptr=U.data_ptr(), B_ptr=Bm.data_ptr(), V_ptr=V.data_ptr(), S_ptr=S.data_ptr(),
                            s_dtype=B.F64, lds=n)
        keep.append((Md, U, Bm, V, S, prob, res))
        tickets.append(ctx.submit(prob, res))
    for t in tickets:
        assert ctx.poll(t, -1) == B.OK
    for a, (_, U, Bm, V, S, _, res) in zip(alone, keep):
        assert res.iters == 8
        assert torch.equal(U, a.U) and torch.equal(S, a.S)


def test_invalid_arguments_are_rejected(ctx):
    Md = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    for kw in (dict(m=0, n=8, r=1), dict(m=8, n=8, r=9), dict(m=8, n=8, r=2, rho=1.0), dict(m=8, n=8, r=70)):
        p = B.make_problem(M_ptr=Md.data_ptr(), m_dtype=B.F64, **kw)
        res = B.make_result()
        assert ctx.solve(p, res) == B.E_INVAL
        assert ctx.last_error()


def test_zero_matrix_is_rejected(ctx):
    Md = torch.zeros((16, 12), dtype=torch.float64, device="cuda")
    p = B.make_problem(m=16, n=12, r=2, M_ptr=Md.data_ptr(), m_dtype=B.F64)
    assert ctx.solve(p, B.make_result()) == B.E_INVAL


def test_rank_deficient_input_reports_rank_error(ctx):
    g = synth.rng(3)
    M = g.standard_normal((40, 2)) @ g.standard_normal((2, 30))
    with pytest.raises(O.RankDeficient):
        O.fr_adm(M, 4, fixed_iters=1)
    Md = torch.from_numpy(M).cuda()
    sol = B.solve_torch(ctx, Md, 4, fixed_iters=1, check=False)
    assert sol.status == B.E_RANK


def test_photometric_stack_mixed_matches_oracle(ctx):
    # the photometric-stereo recipe (Lambertian stack, rank 3, attached shadows, specular
    # outliers, float32 storage) at 64 x 64 pixels x 40 images: tall-skinny, SIMT path
    prob = synth.photometric(side=64, n_images=40, seed=1002)
    M = prob.values_f64()
    ref = O.fr_adm(M, 3, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300)
    for prec, tol in ((B.PREC_FP64, FP64_TOL), (B.PREC_MIXED, MIXED_TOL)):
        sol = B.solve_torch(ctx, _dev(prob), 3, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300, precision=prec)
        assert abs(sol.iters - ref.iters) <= (0 if prec == B.PREC_FP64 else 3)
        assert _rel(_gpu_L(sol), ref.L) <= tol


def test_affinity_nystrom_mixed_matches_oracle(ctx):
    # the spectral-clustering recipe (symmetric block affinity, 20 clusters, bf16) through
    # FR-Nys with l = 10 r = 200 sampled columns (Algorithm 2's k = 10), mixed precision.  The
    # result goes through the pseudo-inverse of the l x l core, whose conditioning (sigma_r /
    # sigma_1 = 0.18 here) scales the block solves' rounding: with l = 128 it is 0.03 and even the
    # float64 path moves L by 3e-6.
    prob = synth.affinity(n=1024, k=20, seed=1003, dtype="bf16")
    M = prob.values_f64()
    perm = synth.row_permutation(1024, 5)
    ref = O.fr_nys(M, 20, 200, perm, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), 20, nys_l=200, nys_perm=torch.from_numpy(perm).cuda(), rho=1.5, mu0=1.0,
                        tol=1e-9, max_iter=300, precision=B.PREC_MIXED, want_L=True)
    assert _rel(sol.L.cpu().numpy(), ref.L) <= MIXED_TOL
