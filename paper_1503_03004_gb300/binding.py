"""ctypes binding of libsfr (include/sfr.h): argument marshalling only.

Every step of the solve runs inside the native library; this module only
loads it, fills the C structs and passes pointers.  PyTorch supplies device
memory and the CUDA stream.  Loading fails loudly when libsfr.so has not been
built: there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfr.so")

# sfr_status
OK, PENDING, E_INVAL, E_NOMEM, E_CUDA, E_RANK, E_NOCONV, E_NAN, E_TIMEOUT, E_BUSY = 0, 1, -1, -2, -3, -4, -5, -6, -7, -8
STATUS_NAMES = {OK: "OK", PENDING: "PENDING", E_INVAL: "E_INVAL", E_NOMEM: "E_NOMEM", E_CUDA: "E_CUDA",
                E_RANK: "E_RANK", E_NOCONV: "E_NOCONV", E_NAN: "E_NAN", E_TIMEOUT: "E_TIMEOUT", E_BUSY: "E_BUSY"}
# sfr_dtype
F64, F32, BF16 = 0, 1, 2
# sfr_precision
PREC_FP64, PREC_MIXED = 0, 1
# sfr_memspace
MEM_DEVICE, MEM_HOST = 0, 1

DTYPE_CODES = {"f64": F64, "f32": F32, "bf16": BF16}


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("profile", ctypes.c_int), ("max_batch", ctypes.c_int)]


# sfr_stat_kind
STAT_SWEEP, STAT_WPASS, STAT_RXR, STAT_ALL, STAT_PPASS, STAT_COUNT = 0, 1, 2, 3, 4, 5


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("timed", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ldm", ctypes.c_int64), ("r", ctypes.c_int32),
                ("m_dtype", ctypes.c_int), ("M", ctypes.c_void_p), ("mu0", ctypes.c_double), ("rho", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("fixed_iters", ctypes.c_int32), ("precision", ctypes.c_int), ("mem", ctypes.c_int),
                ("nys_l", ctypes.c_int32), ("nys_perm", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("B", ctypes.c_void_p), ("V", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("s_dtype", ctypes.c_int), ("lds", ctypes.c_int64), ("L", ctypes.c_void_p),
                ("iters", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("lambda_min_B", ctypes.c_double),
                ("status", ctypes.c_int), ("path", ctypes.c_int32)]


# sfr_path_flag bits of Result.path
PATH_TC = 1


class OptFullProblem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ldm", ctypes.c_int64), ("r", ctypes.c_int32),
                ("m_dtype", ctypes.c_int), ("M", ctypes.c_void_p), ("V0", ctypes.c_void_p), ("B0", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int),
                ("mem", ctypes.c_int)]


class OptFullResult(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("B", ctypes.c_void_p), ("V", ctypes.c_void_p), ("iters", ctypes.c_int32),
                ("rel_change", ctypes.c_double), ("lambda_min_B", ctypes.c_double), ("status", ctypes.c_int)]


# (name, restype, argtypes) of every entry point declared in include/sfr.h
SIGNATURES = [
    ("sfr_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Config)]),
    ("sfr_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(Result)]),
    ("sfr_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(Result),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    ("sfr_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64]),
    ("sfr_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("sfr_solve_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(Result)]),
    ("sfr_fixed_rank_opt_full", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(OptFullProblem),
                                               ctypes.POINTER(OptFullResult)]),
    ("sfr_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KernelStat), ctypes.c_int32, ctypes.c_int32]),
    ("sfr_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("sfr_version", ctypes.c_char_p, []),
]

_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsfr.so (raises if it is missing: the library must be built first)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsfr.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class SfrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Context:
    """An sfr_ctx on one device (sfr_create / sfr_destroy)."""

    def __init__(self, device: int = 0, stream: int | None = None, hbm_budget_bytes: int = 0, max_slots: int = 0,
                 profile: int = 0, max_batch: int = 0):
        """profile: 0 none, 1 (or True) sweep, W pass and r x r kernels timed, 2 the sweep only.
        max_batch > 0: the grouped serving engine for sfr_submit (see include/sfr.h)."""
        self.lib = load()
        self.handle = ctypes.c_void_p()
        cfg = Config(device=device, hbm_budget_bytes=hbm_budget_bytes, max_slots=max_slots,
                     cuda_stream=ctypes.c_void_p(stream) if stream else None, profile=int(profile),
                     max_batch=max_batch)
        st = self.lib.sfr_create(ctypes.byref(self.handle), ctypes.byref(cfg))
        if st != OK:
            raise SfrError(st, self.lib.sfr_last_error(None).decode())

    def last_error(self) -> str:
        return self.lib.sfr_last_error(self.handle).decode()

    def solve(self, prob: Problem, res: Result) -> int:
        return self.lib.sfr_solve(self.handle, ctypes.byref(prob), ctypes.byref(res))

    def solve_noalloc(self, prob: Problem, res: Result) -> int:
        return self.lib.sfr_solve_noalloc(self.handle, ctypes.byref(prob), ctypes.byref(res))

    def opt_full(self, prob: OptFullProblem, res: OptFullResult) -> int:
        return self.lib.sfr_fixed_rank_opt_full(self.handle, ctypes.byref(prob), ctypes.byref(res))

    def submit(self, prob: Problem, res: Result) -> int:
        t = ctypes.c_uint64()
        st = self.lib.sfr_submit(self.handle, ctypes.byref(prob), ctypes.byref(res), ctypes.byref(t))
        if st != OK:
            raise SfrError(st, self.last_error())
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        return self.lib.sfr_poll(self.handle, ticket, timeout_us)

    def stats(self, reset: bool = False) -> list:
        arr = (KernelStat * STAT_COUNT)()
        st = self.lib.sfr_stats(self.handle, arr, STAT_COUNT, int(reset))
        if st != OK:
            raise SfrError(st, self.last_error())
        return [dict(launches=a.launches, timed=a.timed, total_ms=a.total_ms, bytes=a.bytes) for a in arr]

    def close(self):
        if self.handle:
            self.lib.sfr_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_problem(*, m: int, n: int, r: int, M_ptr: int, m_dtype: int, ldm: int | None = None, mu0: float = 1.0,
                 rho: float = 1.5, mu_max: float = 1e9, tol: float = 1e-9, max_iter: int = 500,
                 fixed_iters: int = 0, precision: int = PREC_FP64, mem: int = MEM_DEVICE, nys_l: int = 0,
                 nys_perm_ptr: int = 0) -> Problem:
    return Problem(m=m, n=n, ldm=ldm if ldm is not None else n, r=r, m_dtype=m_dtype, M=M_ptr, mu0=mu0, rho=rho,
                   mu_max=mu_max, tol=tol, max_iter=max_iter, fixed_iters=fixed_iters, precision=precision, mem=mem,
                   nys_l=nys_l, nys_perm=nys_perm_ptr or None)


def make_result(*, U_ptr=0, B_ptr=0, V_ptr=0, S_ptr=0, s_dtype=F64, lds=0, L_ptr=0) -> Result:
    return Result(U=U_ptr or None, B=B_ptr or None, V=V_ptr or None, S=S_ptr or None, s_dtype=s_dtype, lds=lds,
                  L=L_ptr or None, iters=0, rel_residual=0.0, lambda_min_B=0.0, status=PENDING, path=0)


@dataclass
class Solution:
    U: object
    B: object
    V: object
    S: object
    L: object
    iters: int
    rel_residual: float
    lambda_min_B: float
    status: int
    path: int = 0          # PATH_TC bit: the tensor-core sweep and W pass ran


def solve_torch(ctx: Context, M, r: int, *, precision: int = PREC_FP64, want_L: bool = False, s_dtype: int = F64,
                nys_l: int = 0, nys_perm=None, check: bool = True, **kw) -> Solution:
    """Solve with device tensors: M (2-D CUDA tensor, row-major rows; float64/float32/bfloat16).

    Output buffers are allocated with torch on M's device; the library writes them.
    """
    import torch
    assert M.is_cuda and M.dim() == 2 and M.stride(1) == 1
    code = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[M.dtype]
    m, n = M.shape
    dev = M.device
    sd = torch.float64 if s_dtype == F64 else torch.float32
    U = torch.empty((m, r), dtype=torch.float64, device=dev)
    B = torch.empty((r, r), dtype=torch.float64, device=dev)
    V = torch.empty((n, r), dtype=torch.float64, device=dev)
    S = torch.empty((m, n), dtype=sd, device=dev)
    L = torch.empty((m, n), dtype=sd, device=dev) if want_L else None
    perm_ptr = 0
    if nys_l:
        assert nys_perm is not None and nys_perm.is_cuda and nys_perm.dtype == torch.int64
        perm_ptr = nys_perm.data_ptr()
    prob = make_problem(m=m, n=n, r=r, M_ptr=M.data_ptr(), m_dtype=code, ldm=M.stride(0), precision=precision,
                        mem=MEM_DEVICE, nys_l=nys_l, nys_perm_ptr=perm_ptr, **kw)
    res = make_result(U_ptr=U.data_ptr(), B_ptr=B.data_ptr(), V_ptr=V.data_ptr(), S_ptr=S.data_ptr(),
                      s_dtype=s_dtype, lds=n, L_ptr=L.data_ptr() if L is not None else 0)
    torch.cuda.synchronize(dev)
    st = ctx.solve(prob, res)
    if check and st not in (OK,):
        raise SfrError(st, ctx.last_error())
    return Solution(U=U, B=B, V=V, S=S, L=L, iters=res.iters, rel_residual=res.rel_residual,
                    lambda_min_B=res.lambda_min_B, status=st, path=res.path)


@dataclass
class OptFullSolution:
    U: object
    B: object
    V: object
    iters: int
    rel_change: float
    lambda_min_B: float
    status: int


def opt_full_torch(ctx: Context, M, r: int, *, V0=None, B0=None, tol: float = 0.0, max_iter: int = 50,
                   precision: int = PREC_FP64, check: bool = True) -> OptFullSolution:
    """FixedRankOptFull (Algorithm 4) on a device tensor M (2-D CUDA tensor with unit column stride;
    float64/float32/bfloat16).  V0 (n x r) and B0 (r x r) are optional float64 CUDA tensors."""
    import torch
    assert M.is_cuda and M.dim() == 2 and M.stride(1) == 1
    code = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[M.dtype]
    m, n = M.shape
    dev = M.device
    U = torch.empty((m, r), dtype=torch.float64, device=dev)
    B = torch.empty((r, r), dtype=torch.float64, device=dev)
    V = torch.empty((n, r), dtype=torch.float64, device=dev)
    for t, shape in ((V0, (n, r)), (B0, (r, r))):
        assert t is None or (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == shape)
    prob = OptFullProblem(m=m, n=n, ldm=M.stride(0), r=r, m_dtype=code, M=M.data_ptr(),
                          V0=V0.data_ptr() if V0 is not None else None, B0=B0.data_ptr() if B0 is not None else None,
                          tol=tol, max_iter=max_iter, precision=precision, mem=MEM_DEVICE)
    res = OptFullResult(U=U.data_ptr(), B=B.data_ptr(), V=V.data_ptr(), iters=0, rel_change=0.0, lambda_min_B=0.0,
                        status=PENDING)
    torch.cuda.synchronize(dev)
    st = ctx.opt_full(prob, res)
    if check and st != OK:
        raise SfrError(st, ctx.last_error())
    return OptFullSolution(U=U, B=B, V=V, iters=res.iters, rel_change=res.rel_change, lambda_min_B=res.lambda_min_B,
                           status=st)
