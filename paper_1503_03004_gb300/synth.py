"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Every generator draws from numpy's counter-based Philox bit generator, so the
same seed gives bit-identical arrays on x86 and Arm hosts.  Outputs are
row-major, C-contiguous numpy arrays.  The same arrays feed the CPU oracle
and the CUDA library; low-precision storage (float32 / bfloat16) is applied
here, once, so both sides see exactly the same stored values.

Workload recipes (sizes are arguments so tests can run the same recipe small):
  * planted(...)           L0 = U0 V0^T with U0, V0 iid N(0,1); outliers on a
                           Bernoulli(p) support with values uniform in [-a, a].
                           With a = 1 this is the synthetic recipe of the
                           paper's Sec. 5.1 (Tables 1 and 2); with a = 50 it is
                           the 500 x 500 / 16384 x 16384 workloads.
  * photometric(...)       Lambertian image stack (pixels x images) of a
                           smooth random height field, rank 3 before shadows,
                           with attached-shadow zeros and specular outliers
                           (stands in for the photometric-stereo data of Sec. 5.2).
  * affinity(...)          symmetric block affinity of k equal-size clusters
                           with symmetric outliers (stands in for the
                           spectral-clustering data of Sec. 5.3).
  * request_stream(...)    uneven (m, n, r, p) decomposition requests with
                           Poisson arrival times.
  * row_permutation(...)   the random row shuffle FR-Nys draws (Algorithm 2).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); return the uint16 bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    """Exact float64 values of bfloat16 bit patterns."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@dataclasses.dataclass
class Problem:
    """One stored input matrix plus what was planted in it (when known)."""
    M: np.ndarray                 # stored values: float64, float32 or uint16 (bfloat16 bits)
    dtype: str                    # "f64" | "f32" | "bf16"
    r: int
    U0: np.ndarray | None = None  # planted factors (float64), L0 = U0 @ V0.T
    V0: np.ndarray | None = None
    S0_mask: np.ndarray | None = None  # planted outlier support (bool), None if not sparse
    name: str = ""

    @property
    def shape(self):
        return self.M.shape

    def values_f64(self) -> np.ndarray:
        """The exact stored values as float64 (what the oracle must see)."""
        if self.dtype == "bf16":
            return bf16_bits_to_f64(self.M)
        return self.M.astype(np.float64)


def _store(A64: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "f64":
        return np.ascontiguousarray(A64, dtype=np.float64)
    if dtype == "f32":
        return np.ascontiguousarray(A64, dtype=np.float32)
    if dtype == "bf16":
        return to_bf16_bits(np.asarray(A64, dtype=np.float32))
    raise ValueError(dtype)


def planted(m: int, n: int, r: int, *, p: float, amp: float, seed: int,
            dtype: str = "f64", name: str = "") -> Problem:
    """M = U0 V0^T + S0; U0, V0 ~ N(0,1); S0 ~ Bernoulli(p) support, values U[-amp, amp]."""
    g = rng(seed)
    U0 = g.standard_normal((m, r))
    V0 = g.standard_normal((n, r))
    mask = g.random((m, n), dtype=np.float32) < p
    vals = g.uniform(-amp, amp, size=(m, n)).astype(np.float32 if dtype != "f64" else np.float64)
    if dtype == "f64":
        L0 = U0 @ V0.T
        M = L0 + np.where(mask, vals, 0.0)
    else:
        L0 = U0.astype(np.float32) @ V0.T.astype(np.float32)
        M = L0 + np.where(mask, vals, np.float32(0.0))
    return Problem(M=_store(M, dtype), dtype=dtype, r=r, U0=U0, V0=V0, S0_mask=mask,
                   name=name or f"planted_{m}x{n}_r{r}")


def square_fp64_500(seed: int = 1000) -> Problem:
    """500 x 500, r = 25, 10% outliers in [-50, 50], float64 storage."""
    return planted(500, 500, 25, p=0.10, amp=50.0, seed=seed, dtype="f64", name="square500_r25_f64")


def paper_table1(m: int, r: int = 10, seed: int = 7) -> Problem:
    """Sec. 5.1 recipe: L = A B^T, A, B ~ N(0,1); 10% outliers with magnitudes in [-1, 1]."""
    return planted(m, m, r, p=0.10, amp=1.0, seed=seed, dtype="f64", name=f"paper_table1_{m}_r{r}")


def square_large(m: int = 16384, r: int = 64, dtype: str = "bf16", seed: int = 1001) -> Problem:
    """16384 x 16384, r = 64, 5% outliers in [-50, 50]; float32 or bfloat16 storage."""
    return planted(m, m, r, p=0.05, amp=50.0, seed=seed, dtype=dtype, name=f"square{m}_r{r}_{dtype}")


def photometric(side: int = 1024, n_images: int = 40, *, p_spec: float = 0.10, seed: int = 1002,
                n_bumps: int = 16) -> Problem:
    """Lambertian stack: pixels (side^2) x images, rank 3 before attached shadows.

    Height field = sum of Gaussian bumps; normals by central differences;
    albedo ~ U[0.2, 1]; light directions uniform on the upper hemisphere with
    elevation >= 15 degrees; M = albedo * max(0, n.l) plus additive U[0, 1]
    specular outliers on a Bernoulli(p_spec) support; float32 storage.
    The planted factors are the signed shading albedo * (n.l) (before the
    shadow clamp), so M - L0 is not sparse: this workload is checked against
    the oracle, not against L0.
    """
    g = rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, side), np.linspace(0, 1, side), indexing="ij")
    h = np.zeros((side, side))
    for _ in range(n_bumps):
        cx, cy = g.uniform(0.1, 0.9, 2)
        s = g.uniform(0.05, 0.2)
        a = g.uniform(-0.3, 0.3)
        h += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    hy, hx = np.gradient(h, 1.0 / (side - 1))
    N = np.stack([-hx, -hy, np.ones_like(h)], axis=-1).reshape(-1, 3)
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    albedo = g.uniform(0.2, 1.0, size=N.shape[0])
    el = np.arcsin(g.uniform(np.sin(np.deg2rad(15.0)), 1.0, n_images))
    az = g.uniform(0, 2 * np.pi, n_images)
    Ldir = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
    U0 = N * albedo[:, None]                   # pixels x 3
    V0 = Ldir                                  # images x 3
    shade = np.maximum(0.0, U0 @ V0.T)
    mask = g.random(shade.shape, dtype=np.float32) < p_spec
    spec = g.uniform(0.0, 1.0, size=shade.shape)
    M = np.where(mask, shade + spec, shade)
    return Problem(M=_store(M, "f32"), dtype="f32", r=3, U0=U0, V0=V0, S0_mask=None,
                   name=f"photometric_{side * side}x{n_images}_r3")


AFFINITY_TILE = 2048


def _affinity_tile(seed: int, bi: int, bj: int, rows: int, cols: int, p_out: float):
    """Draws of the upper-triangle tile (bi, bj), bi <= bj, from its own Philox stream: standard
    normal noise, the outlier mask and the outlier values (U[0, 1])."""
    g = np.random.Generator(np.random.Philox(key=int(seed), counter=[0, 0, int(bi), int(bj)]))
    z = g.standard_normal((rows, cols))
    hit = g.random((rows, cols), dtype=np.float32) < p_out
    val = g.random((rows, cols))
    return z, hit, val


def affinity_rows(n: int, k: int, i0: int, i1: int, *, p_out: float = 0.03, seed: int = 1003):
    """Rows [i0, i1) of the affinity recipe in float64 (see `affinity`), plus the outlier mask of
    those rows.  Memory is O((i1 - i0) n): tiles of the upper triangle are drawn from their own
    streams, and a lower tile is the mirror of its upper tile."""
    labels = affinity_labels(n, k, seed)
    T = AFFINITY_TILE
    A = np.empty((i1 - i0, n))
    M = np.zeros((i1 - i0, n), dtype=bool)
    for bi in range(i0 // T, (i1 - 1) // T + 1):
        r0, r1 = bi * T, min(n, (bi + 1) * T)
        for bj in range(n // T + (n % T > 0)):
            c0, c1 = bj * T, min(n, (bj + 1) * T)
            if bi <= bj:
                z, hit, val = _affinity_tile(seed, bi, bj, r1 - r0, c1 - c0, p_out)
                if bi == bj:  # diagonal tile: mirror its strict upper part, no outliers on the diagonal
                    up = np.triu(np.ones((r1 - r0, c1 - c0), dtype=bool), 1)
                    d = np.diag(z).copy()
                    z = np.where(up, z, 0.0)
                    z = z + z.T + np.diag(d)
                    hit = hit & up
                    val = np.where(hit, val, 0.0)
                    hit = hit | hit.T
                    val = val + val.T
            else:  # lower tile: transpose of the upper tile (bj, bi)
                z, hit, val = _affinity_tile(seed, bj, bi, c1 - c0, r1 - r0, p_out)
                z, hit, val = z.T, hit.T, val.T
            same = labels[r0:r1, None] == labels[None, c0:c1]
            tile = np.where(same, 0.8 + 0.05 * z, 0.05 + 0.02 * z) + np.where(hit, val, 0.0)
            a0, a1 = max(i0, r0), min(i1, r1)
            A[a0 - i0:a1 - i0, c0:c1] = tile[a0 - r0:a1 - r0]
            M[a0 - i0:a1 - i0, c0:c1] = hit[a0 - r0:a1 - r0]
    return A, M


def affinity_labels(n: int, k: int, seed: int) -> np.ndarray:
    """Cluster labels of the affinity recipe: k clusters whose sizes differ by at most one,
    assigned to the nodes in a random order."""
    sizes = np.full(k, n // k)
    sizes[: n % k] += 1
    return rng(seed).permutation(np.repeat(np.arange(k), sizes))


def affinity(n: int = 32768, k: int = 20, *, p_out: float = 0.03, seed: int = 1003,
             dtype: str = "bf16") -> Problem:
    """Symmetric n x n affinity of k clusters (sizes differ by at most one, labels shuffled).

    Within-cluster 0.8 + N(0, 0.05^2), across 0.05 + N(0, 0.02^2) (noise mirrored across the
    diagonal), plus 3% symmetric additive outliers U[0, 1] off the diagonal.  Generated row block
    by row block (`affinity_rows`), so the host holds one float64 block at a time plus the stored
    matrix (2 GB at n = 32768 in bfloat16).
    """
    labels = affinity_labels(n, k, seed)
    out = np.empty((n, n), dtype=np.float64 if dtype == "f64" else np.float32 if dtype == "f32" else np.uint16)
    mask = np.zeros((n, n), dtype=bool) if n <= 8192 else None
    T = AFFINITY_TILE

    def block(i0):
        A, hit = affinity_rows(n, k, i0, min(n, i0 + T), p_out=p_out, seed=seed)
        out[i0:i0 + T] = _store(A, dtype)
        if mask is not None:
            mask[i0:i0 + T] = hit

    # row blocks are independent (each draws its tiles from their own streams): a few threads
    # (numpy releases the GIL in its generators and element-wise kernels), same bits in any order
    import concurrent.futures
    with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
        list(ex.map(block, range(0, n, T)))
    Z = np.zeros((n, k))
    Z[np.arange(n), labels] = 1.0
    return Problem(M=out, dtype=dtype, r=k, U0=Z, V0=None, S0_mask=mask, name=f"affinity_{n}_k{k}_{dtype}")


def row_permutation(m: int, seed: int) -> np.ndarray:
    """Random row shuffle drawn by FR-Nys (Algorithm 2); int64, shuffled row i = input row perm[i]."""
    return rng(seed).permutation(m).astype(np.int64)


@dataclasses.dataclass
class Request:
    arrival_s: float
    m: int
    n: int
    r: int
    p: float
    seed: int


def request_stream(count: int = 4096, *, rate_per_s: float = 1000.0, seed: int = 1004,
                   m_range=(256, 8192), n_range=(16, 512), ranks=(3, 5, 10, 25)) -> list:
    """Poisson arrivals of uneven decomposition requests.

    m ~ U[m_range], n ~ U[n_range], r from `ranks` restricted to r <= n/2
    (redrawn from the admissible subset), outlier fraction ~ U[0.02, 0.15].
    """
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate_per_s, count))
    out = []
    for i in range(count):
        m = int(g.integers(m_range[0], m_range[1] + 1))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        ok = [r for r in ranks if r <= n // 2]
        r = int(ok[int(g.integers(0, len(ok)))])
        p = float(g.uniform(0.02, 0.15))
        out.append(Request(arrival_s=float(t[i]), m=m, n=n, r=r, p=p, seed=int(seed * 100003 + i)))
    return out
