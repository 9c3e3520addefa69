"""GPU parity at the workloads' full sizes.

The float64 oracle cannot run inside a test at these sizes, so its results come as seeded
samples written by `tests/golden/make_fullsize_samples.py` (which calls only `oracle/` and
the input generators): the oracle's iteration count and its L_ij, S_ij at 4096 positions.
The GPU side is the same C-ABI call `bench.py` times.  Bars as in test_gpu_parity: 1e-9
relative on L for the float64 path, 1e-5 for the mixed path (S: 1e-4).  Where the oracle is
cheap enough (the Nystrom workload at 8192, l = 512) it runs in the test itself.
"""
import os

import numpy as np
import pytest

from oracle import fradm as O
from paper_1503_03004_gb300 import binding as B
from paper_1503_03004_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _golden(name):
    meta, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 2:
                meta[parts[0]] = float(parts[1])
            else:
                rows.append([float(x) for x in parts])
    a = np.array(rows)
    return meta, a[:, 0].astype(np.int64), a[:, 1].astype(np.int64), a[:, 2], a[:, 3], a[:, 4]


def _dev(prob):
    if prob.dtype == "bf16":
        return torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(prob.M).cuda()


def _sampled_L(sol, ii, jj):
    U = sol.U.cpu().numpy()
    V = sol.V.cpu().numpy()
    Bm = sol.B.cpu().numpy()
    return np.einsum("ka,ab,kb->k", U[ii], Bm, V[jj])


def _sampled_S(sol, ii, jj):
    it = torch.from_numpy(ii).to(sol.S.device)
    jt = torch.from_numpy(jj).to(sol.S.device)
    return sol.S[it, jt].double().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _invariants(sol, tol):
    r = sol.B.shape[0]
    eye = torch.eye(r, dtype=torch.float64, device=sol.U.device)
    assert float((sol.U.T @ sol.U - eye).abs().max()) <= tol
    assert float((sol.V.T @ sol.V - eye).abs().max()) <= tol
    assert float((sol.B - sol.B.T).abs().max()) <= 1e-12 * float(sol.B.abs().max())
    assert sol.lambda_min_B > 0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_photometric_full_size_matches_oracle_samples(ctx, precision):
    # 1024 x 1024 pixels x 40 images, rank 3, float32 storage (the photometric-stereo workload)
    meta, ii, jj, L_ref, S_ref, z_ref = _golden("photometric_1048576x40_r3_samples.txt")
    prob = synth.photometric(side=1024, n_images=40, seed=1002)
    prec = B.PREC_MIXED if precision == "mixed" else B.PREC_FP64
    sol = B.solve_torch(ctx, _dev(prob), 3, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300, precision=prec,
                        s_dtype=B.F32 if precision == "mixed" else B.F64)
    assert sol.status == B.OK and sol.rel_residual <= 1e-9
    L = _sampled_L(sol, ii, jj)
    S = _sampled_S(sol, ii, jj)
    if precision == "fp64":
        assert sol.iters == int(meta["iters"])
        assert _rel(L, L_ref) <= 1e-9
        thr = 1.0 / meta["mu_last"]
        near = np.abs(np.abs(z_ref) - thr) <= 1e-9 * max(1.0, np.abs(z_ref).max())
        assert np.count_nonzero(((S != 0) != (S_ref != 0)) & ~near) == 0
        _invariants(sol, 1e-10)
    else:
        assert abs(sol.iters - int(meta["iters"])) <= 3
        assert _rel(L, L_ref) <= 1e-5
        _invariants(sol, 1e-5)


def test_square16384_r64_bf16_mixed_full_size_matches_oracle_samples(ctx):
    # the benchmark workload, through the same call and precision bench.py times
    path = os.path.join(GOLDEN, "square16384_r64_bf16_samples.txt")
    if not os.path.exists(path):
        pytest.skip("oracle samples for the 16384 x 16384 workload not generated")
    meta, ii, jj, L_ref, S_ref, _ = _golden("square16384_r64_bf16_samples.txt")
    prob = synth.square_large(16384, 64, dtype="bf16", seed=1001)
    sol = B.solve_torch(ctx, _dev(prob), 64, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300, precision=B.PREC_MIXED,
                        s_dtype=B.F32)
    assert sol.status == B.OK and sol.rel_residual <= 1e-9
    L = _sampled_L(sol, ii, jj)
    S = _sampled_S(sol, ii, jj)
    assert _rel(L, L_ref) <= 1e-5
    assert _rel(S, S_ref) <= 1e-4
    _invariants(sol, 1e-5)
    # The float64 path takes the oracle's 41 iterations here; the mixed path's residual
    # ||M - L - S|| / ||M|| falls by about 1/rho per iteration near the end (float32 / bfloat16
    # rounding of the iterates), so it reaches 1e-9 four iterations later.
    assert 0 <= sol.iters - int(meta["iters"]) <= 4


def test_square16384_r64_f32_fp64_full_size_matches_oracle_samples(ctx):
    # the 16384 x 16384 rank-64 recipe stored in float32, solved on the float64 path
    path = os.path.join(GOLDEN, "square16384_r64_f32_samples.txt")
    if not os.path.exists(path):
        pytest.skip("oracle samples for the 16384 x 16384 float32 workload not generated")
    meta, ii, jj, L_ref, S_ref, z_ref = _golden("square16384_r64_f32_samples.txt")
    prob = synth.square_large(16384, 64, dtype="f32", seed=1001)
    sol = B.solve_torch(ctx, _dev(prob), 64, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300, precision=B.PREC_FP64,
                        s_dtype=B.F64)
    assert sol.status == B.OK and sol.rel_residual <= 1e-9
    assert sol.iters == int(meta["iters"])
    L = _sampled_L(sol, ii, jj)
    S = _sampled_S(sol, ii, jj)
    assert _rel(L, L_ref) <= 1e-9
    thr = 1.0 / meta["mu_last"]
    near = np.abs(np.abs(z_ref) - thr) <= 1e-9 * max(1.0, np.abs(z_ref).max())
    assert np.count_nonzero(((S != 0) != (S_ref != 0)) & ~near) == 0
    assert np.linalg.norm(S - S_ref) <= 1e-9 * np.linalg.norm(L_ref)
    _invariants(sol, 1e-10)


def test_affinity_nystrom_32768_full_size_matches_oracle_samples(ctx):
    # the spectral-clustering workload at its full size: n = 32768, 20 clusters, bf16, FR-Nys with
    # l = 2048 on the mixed path (the call bench.py --config affinity_32768_r20_nys2048 times)
    path = os.path.join(GOLDEN, "affinity_32768_r20_nys2048_samples.txt")
    if not os.path.exists(path):
        pytest.skip("oracle samples for the 32768^2 affinity workload not generated")
    meta, ii, jj, L_ref, S_ref, _ = _golden("affinity_32768_r20_nys2048_samples.txt")
    prob = synth.affinity(n=32768, k=20, seed=1003, dtype="bf16")
    Md = _dev(prob)
    del prob
    perm = torch.from_numpy(synth.row_permutation(32768, 5)).cuda()
    sol = B.solve_torch(ctx, Md, 20, nys_l=2048, nys_perm=perm, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300,
                        precision=B.PREC_MIXED, s_dtype=B.F32, want_L=True)
    assert sol.status == B.OK
    assert abs(sol.iters - int(meta["iters"])) <= 8
    it = torch.from_numpy(ii).cuda()
    jt = torch.from_numpy(jj).cuda()
    L = sol.L[it, jt].double().cpu().numpy()
    S = sol.S[it, jt].double().cpu().numpy()
    assert _rel(L, L_ref) <= 1e-5
    assert np.linalg.norm(S - S_ref) <= 1e-5 * np.linalg.norm(L_ref)


def test_affinity_nystrom_8192_matches_oracle(ctx):
    # the spectral-clustering workload through FR-Nys at n = 8192 with l = 512 (the full
    # workload's l / n = 2048 / 32768); the oracle runs here (about 30 s)
    prob = synth.affinity(n=8192, k=20, seed=1003, dtype="bf16")
    perm = synth.row_permutation(8192, 5)
    ref = O.fr_nys(prob.values_f64(), 20, 512, perm, rho=1.5, mu0=1.0, tol=1e-9, max_iter=300)
    sol = B.solve_torch(ctx, _dev(prob), 20, nys_l=512, nys_perm=torch.from_numpy(perm).cuda(), rho=1.5, mu0=1.0,
                        tol=1e-9, max_iter=300, precision=B.PREC_MIXED, want_L=True)
    assert sol.status == B.OK
    assert _rel(sol.L.cpu().numpy().astype(np.float64), ref.L) <= 1e-5
