"""ctypes binding of libhssnd.so (the C ABI in include/hssnd.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  There
is no CPU fallback: importing this module fails loudly when the library is
missing, and every call raises HssError on a non-zero return code.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhssnd.so")

HSS_OK, HSS_EINVAL, HSS_ENOMEM, HSS_ESINGULAR, HSS_ENOCONV, HSS_ETIMEOUT, HSS_ECUDA = range(7)
SCHEMES = {"box": 0, "hslab": 1, "vslab": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}
CAP_POLICIES = {"keep": 0, "accept": 1}

EXPORTED = [
    "hss_nd_opts_default", "hss_factor_opts_default", "fgmres_opts_default",
    "nd_order", "hss_tree_info", "hss_tree_export", "hss_factor", "hss_factor_get_info",
    "hss_factor_export_front", "hss_apply", "hss_spmv", "fgmres_solve", "fgmres_history",
    "hss_tree_destroy", "hss_factor_destroy", "hss_last_error",
    "hss_launch_count", "hss_profile_enable", "hss_profile_reset", "hss_profile_read", "hss_gemm_f32",
    "hss_gemm_f32_static", "nd_order_batched", "hss_factor_batched", "fgmres_solve_batched",
    "hss_rank_features", "hss_rank_model_create", "hss_rank_model_destroy", "hss_rank_model_get",
    "hss_rank_model_set", "hss_rank_model_fit_norm", "hss_rank_model_loss_grad", "hss_rank_model_train",
    "hss_rank_model_predict", "hss_factor_export_log", "ilu0_factor", "ilu0_apply", "fgmres_solve_ilu0",
    "ilu0_destroy", "hss_factor_apply_plan", "hss_alloc_count", "hss_tc_timeout_selftest",
    "hss_front_eliminate", "hss_front_compress", "hss_gemm_tuner_read",
]


class HssError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libhssnd error {code}: {msg}")
        self.code = code


class hss_bsr(C.Structure):
    _fields_ = [("nb", C.c_int), ("bs", C.c_int), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p)]


class hss_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("p", C.c_int)]


class hss_nd_opts(C.Structure):
    _fields_ = [("leaf_max", C.c_int), ("scheme", C.c_int)]


class hss_factor_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("compress", C.c_int), ("r0", C.c_int), ("dr", C.c_int),
                ("rmax", C.c_int), ("oversample", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64), ("keep_schur", C.c_int), ("tensor_cores", C.c_int), ("r_init", C.c_void_p),
                ("cap_policy", C.c_int), ("autotune", C.c_int), ("probe", C.c_int), ("sample_bf16", C.c_int),
                ("merge", C.c_int)]


class fgmres_opts(C.Structure):
    _fields_ = [("restart", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int)]


class fgmres_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("max_iters", C.c_int), ("relres", C.c_double), ("converged", C.c_int)]


class hss_tree_desc(C.Structure):
    _fields_ = [("ndof", C.c_int), ("nbox", C.c_int), ("maxlev", C.c_int), ("iset_len", C.c_int),
                ("bset_len", C.c_int), ("bs", C.c_int)]


class hss_factor_info(C.Structure):
    _fields_ = [("factor_bytes", C.c_double), ("front_flops", C.c_double), ("executed_flops", C.c_double),
                ("max_rank", C.c_int), ("max_r", C.c_int), ("rounds", C.c_int), ("nfronts", C.c_int),
                ("capped_fronts", C.c_int), ("probe_regrown", C.c_int), ("gemm_simt", C.c_long),
                ("gemm_tma", C.c_long), ("gemm_staged", C.c_long), ("gemm_timed", C.c_long),
                ("gemm_bf16", C.c_long), ("host_syncs", C.c_long), ("host_sync_ms", C.c_double),
                ("host_ms", C.c_double), ("host_gap_ms", C.c_double)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = C.CDLL(path)
    P = C.c_void_p
    ip = C.POINTER(C.c_int)
    dp = C.POINTER(C.c_double)
    sig = {
        "nd_order": (C.c_int, [C.POINTER(hss_mesh), C.POINTER(hss_bsr), C.POINTER(hss_nd_opts), P, C.POINTER(P)]),
        "hss_tree_info": (C.c_int, [P, C.POINTER(hss_tree_desc)]),
        "hss_tree_export": (C.c_int, [P] + [ip] * 13),
        "hss_factor": (C.c_int, [C.POINTER(hss_bsr), P, C.POINTER(hss_factor_opts), P, C.POINTER(P)]),
        "hss_factor_get_info": (C.c_int, [P, C.POINTER(hss_factor_info)]),
        "hss_factor_export_front": (C.c_int, [P, C.c_int, dp, dp, ip, ip]),
        "hss_apply": (C.c_int, [P, C.c_int, P, C.c_int, P, C.c_int, P]),
        "hss_spmv": (C.c_int, [C.POINTER(hss_bsr), C.c_int, P, C.c_int, P, C.c_int, P]),
        "fgmres_solve": (C.c_int, [C.POINTER(hss_bsr), P, C.c_int, P, C.c_int, P, C.c_int,
                                   C.POINTER(fgmres_opts), C.POINTER(fgmres_stats), P]),
        "fgmres_history": (C.c_int, [C.c_int, dp, C.c_int]),
        "hss_tree_destroy": (None, [P]),
        "hss_factor_destroy": (None, [P]),
        "hss_last_error": (C.c_char_p, []),
        "hss_nd_opts_default": (None, [C.POINTER(hss_nd_opts)]),
        "hss_factor_opts_default": (None, [C.POINTER(hss_factor_opts)]),
        "fgmres_opts_default": (None, [C.POINTER(fgmres_opts)]),
        "hss_launch_count": (C.c_long, []),
        "hss_alloc_count": (C.c_long, []),
        "hss_gemm_tuner_read": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), ip, C.POINTER(C.c_float),
                                          C.POINTER(C.c_float)]),
        "hss_front_eliminate": (C.c_int, [C.c_int, C.c_int, P, C.c_int, C.c_int, C.c_int, P, C.c_int, P, P]),
        "hss_front_compress": (C.c_int, [P, C.c_int, P, C.c_int, C.POINTER(hss_factor_opts), P, C.c_int, ip, ip, ip,
                                         P]),
        "hss_tc_timeout_selftest": (C.c_int, [C.c_long, P]),
        "hss_gemm_f32": (C.c_int, [C.c_int, C.c_int, C.c_int, P, C.c_int, P, C.c_int, P, C.c_int, C.c_float,
                                   C.c_float, C.c_int, P]),
        "hss_gemm_f32_static": (C.c_int, [C.c_int, C.c_int, C.c_int, P, C.c_int, P, C.c_int, P, C.c_int,
                                          C.c_float, C.c_float, C.c_int, P]),
        "nd_order_batched": (C.c_int, [C.c_int, C.POINTER(hss_mesh), C.POINTER(hss_bsr), C.POINTER(hss_nd_opts), P,
                                       C.POINTER(P)]),
        "hss_factor_batched": (C.c_int, [C.c_int, C.POINTER(hss_bsr), P, C.POINTER(hss_factor_opts), P,
                                         C.POINTER(P)]),
        "fgmres_solve_batched": (C.c_int, [P, C.c_int, P, C.c_int, P, C.c_int, C.POINTER(fgmres_opts),
                                           C.POINTER(fgmres_stats), P]),
        "hss_rank_features": (C.c_int, [P, P, C.c_double, P]),
        "hss_rank_model_create": (C.c_int, [C.c_uint64, C.POINTER(P)]),
        "hss_rank_model_destroy": (None, [P]),
        "hss_rank_model_get": (C.c_int, [P, P, P]),
        "hss_rank_model_set": (C.c_int, [P, P, P]),
        "hss_rank_model_fit_norm": (C.c_int, [P, C.c_int, P, P, P]),
        "hss_rank_model_loss_grad": (C.c_int, [P, C.c_int, P, P, C.POINTER(C.c_float), P, P]),
        "hss_rank_model_train": (C.c_int, [P, C.c_int, P, P, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                           C.POINTER(C.c_float), P]),
        "hss_rank_model_predict": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int, P, P, P]),
        "hss_factor_export_log": (C.c_int, [P, C.c_int, ip, ip, ip, ip]),
        "ilu0_factor": (C.c_int, [C.POINTER(hss_bsr), P, C.POINTER(P)]),
        "ilu0_apply": (C.c_int, [P, C.c_int, P, C.c_int, P, C.c_int, P]),
        "fgmres_solve_ilu0": (C.c_int, [C.POINTER(hss_bsr), P, C.c_int, P, C.c_int, P, C.c_int,
                                        C.POINTER(fgmres_opts), C.POINTER(fgmres_stats), P]),
        "ilu0_destroy": (None, [P]),
        "hss_factor_apply_plan": (C.c_int, [P, C.c_int, ip, ip]),
        "hss_profile_enable": (C.c_int, [C.c_int]),
        "hss_profile_reset": (C.c_int, []),
        "hss_profile_read": (C.c_int, [C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_long), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


def _check(rc, allow=()):
    if rc != HSS_OK and rc not in allow:
        raise HssError(rc, _lib.hss_last_error().decode())
    return rc


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


class DeviceBSR:
    """Block-sparse matrix resident on the GPU (int32 structure, fp64 values)."""

    def __init__(self, nb, bs, row_ptr, col_idx, val, device="cuda"):
        self.nb, self.bs = int(nb), int(bs)
        self.row_ptr = torch.as_tensor(np.asarray(row_ptr, dtype=np.int32), device=device)
        self.col_idx = torch.as_tensor(np.asarray(col_idx, dtype=np.int32), device=device)
        self.val = torch.as_tensor(np.ascontiguousarray(val, dtype=np.float64).reshape(-1), device=device)
        self.c = hss_bsr(self.nb, self.bs, self.row_ptr.data_ptr(), self.col_idx.data_ptr(), self.val.data_ptr())

    @classmethod
    def from_host(cls, A, device="cuda"):
        return cls(A.nb, A.bs, A.row_ptr, A.col_idx, A.val, device)

    @property
    def n(self):
        return self.nb * self.bs


def _colmajor(x: torch.Tensor, N: int):
    """(N,) or (N, k) fp64 CUDA tensor -> contiguous (k, N) storage (column-major N x k)."""
    if x.dim() == 1:
        x = x.reshape(N, 1)
    if x.shape[0] != N:
        raise ValueError(f"expected {N} rows, got {tuple(x.shape)}")
    return x.t().contiguous().to(torch.float64), x.shape[1]


class Tree:
    def __init__(self, handle, mesh):
        self.h = C.c_void_p(handle)
        self.mesh = mesh
        self.ninst = 1
        d = hss_tree_desc()
        _check(_lib.hss_tree_info(self.h, C.byref(d)))
        self.desc = d

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hss_tree_destroy(self.h)
            self.h = None

    def export(self) -> dict:
        d = self.desc
        nb_ = d.nbox
        arrs = {k: np.zeros(nb_, dtype=np.int32) for k in
                ("level", "parent", "child0", "child1", "ni", "nb", "ioff", "boff")}
        arrs["lohi"] = np.zeros(6 * nb_, dtype=np.int32)
        arrs["iset"] = np.zeros(max(d.iset_len, 1), dtype=np.int32)
        arrs["bset"] = np.zeros(d.bset_len, dtype=np.int32)
        arrs["fmap"] = np.zeros(d.bset_len, dtype=np.int32)
        arrs["perm"] = np.zeros(d.ndof, dtype=np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))  # noqa: E731
        _check(_lib.hss_tree_export(self.h, *[ip(arrs[k]) for k in (
            "level", "parent", "child0", "child1", "ni", "nb", "ioff", "boff", "lohi", "iset", "bset", "fmap",
            "perm")]))
        arrs["iset"] = arrs["iset"][: d.iset_len]
        arrs["lohi"] = arrs["lohi"].reshape(nb_, 6)
        return arrs


class Factor:
    def __init__(self, handle, tree, precision):
        self.h = C.c_void_p(handle)
        self.tree = tree          # keeps the tree alive
        self.precision = precision

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hss_factor_destroy(self.h)
            self.h = None

    def info(self) -> dict:
        i = hss_factor_info()
        _check(_lib.hss_factor_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in hss_factor_info._fields_}

    def export_log(self) -> dict:
        n = _lib.hss_factor_export_log(self.h, 0, None, None, None, None)
        arrs = {k: np.zeros(max(n, 1), dtype=np.int32) for k in ("box", "kmax", "r", "rounds")}
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))  # noqa: E731
        _lib.hss_factor_export_log(self.h, n, *[ip(arrs[k]) for k in ("box", "kmax", "r", "rounds")])
        return {k: v[:n] for k, v in arrs.items()}

    def apply_plan(self) -> tuple:
        """Columns per work item of each apply stage: (forward, backward) arrays."""
        n = _lib.hss_factor_apply_plan(self.h, 0, None, None)
        if n < 0:
            _check(-n)
        fw, bw = np.zeros(max(n, 1), np.int32), np.zeros(max(n, 1), np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))  # noqa: E731
        _lib.hss_factor_apply_plan(self.h, n, ip(fw), ip(bw))
        return fw[:n], bw[:n]

    def export_front(self, box: int):
        if getattr(self, "_nb", None) is None:
            self._nb = self.tree.export()["nb"]
        nb_ = int(self._nb[box])
        S = np.zeros((nb_, nb_), order="F")
        H = np.zeros((nb_, nb_), order="F")
        kmax, r = C.c_int(0), C.c_int(0)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        _check(_lib.hss_factor_export_front(self.h, box, dp(S), dp(H), C.byref(kmax), C.byref(r)))
        return S, H, kmax.value, r.value


def nd_order(mesh, A: DeviceBSR, leaf_max=64, scheme="box", stream=None) -> Tree:
    """mesh: (dim, (nx, ny[, nz]), p)."""
    dim, n, p = mesh
    n3 = list(n) + [1] * (3 - len(n))
    m = hss_mesh(dim, (C.c_int * 3)(*n3), p)
    o = hss_nd_opts(leaf_max, SCHEMES[scheme])
    out = C.c_void_p()
    _check(_lib.nd_order(C.byref(m), C.byref(A.c), C.byref(o), _stream(stream), C.byref(out)))
    return Tree(out.value, mesh)


def factor_opts(**kw) -> hss_factor_opts:
    o = hss_factor_opts()
    _lib.hss_factor_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "cap_policy" and isinstance(v, str):
            v = CAP_POLICIES[v]
        setattr(o, k, v)
    return o


def hss_factor(A: DeviceBSR, tree: Tree, stream=None, **kw) -> Factor:
    r_init = kw.pop("r_init", None)
    o = factor_opts(**kw)
    if r_init is not None:
        r_init = np.ascontiguousarray(r_init, dtype=np.int32)
        assert r_init.size == tree.desc.nbox
        o.r_init = r_init.ctypes.data
    out = C.c_void_p()
    _check(_lib.hss_factor(C.byref(A.c), tree.h, C.byref(o), _stream(stream), C.byref(out)))
    return Factor(out.value, tree, o.precision)


def front_eliminate(F: np.ndarray, ni: int, precision="fp64", tensor_cores=0, stream=None):
    """hss_front_eliminate on a dense front (HOST array n x n): returns the
    transformed front [F_ii^-1 P^t, W; -F_bi F_ii^-1 P^t, S], the I row of
    each of its first ni columns, and the return code (HSS_OK or
    HSS_ESINGULAR; other codes raise)."""
    Fc = np.asfortranarray(F, dtype=np.float64)
    n = Fc.shape[0]
    out = np.zeros((n, n), dtype=np.float64, order="F")
    perm = np.zeros(max(ni, 1), dtype=np.int32)
    prec = PRECISIONS[precision] if isinstance(precision, str) else precision
    rc = _lib.hss_front_eliminate(n, ni, Fc.ctypes.data, n, prec, tensor_cores, out.ctypes.data, n,
                                  perm.ctypes.data, _stream(stream))
    if rc not in (HSS_OK, HSS_ESINGULAR):
        _check(rc)
    return out, perm[:ni], rc


def front_compress(tree: Tree, box: int, S: np.ndarray, stream=None, **kw):
    """hss_front_compress: the HSS approximant of S (HOST nb x nb) as
    hss_factor builds it for `box`; returns (H, kmax, r, rounds)."""
    r_init = kw.pop("r_init", None)
    o = factor_opts(**kw)
    if r_init is not None:
        r_init = np.ascontiguousarray(r_init, dtype=np.int32)
        assert r_init.size == tree.desc.nbox
        o.r_init = r_init.ctypes.data
    Sc = np.asfortranarray(S, dtype=np.float64)
    nb = Sc.shape[0]
    H = np.zeros((nb, nb), dtype=np.float64, order="F")
    k, r, rounds = C.c_int(), C.c_int(), C.c_int()
    _check(_lib.hss_front_compress(tree.h, box, Sc.ctypes.data, max(nb, 1), C.byref(o), H.ctypes.data, max(nb, 1),
                                   C.byref(k), C.byref(r), C.byref(rounds), _stream(stream)))
    return H, k.value, r.value, rounds.value


def hss_apply(F: Factor, x: torch.Tensor, stream=None) -> torch.Tensor:
    N = F.tree.desc.ndof
    xs, k = _colmajor(x, N)
    ys = torch.empty_like(xs)
    _check(_lib.hss_apply(F.h, k, _ptr(xs), N, _ptr(ys), N, _stream(stream)))
    y = ys.t()
    return y.reshape(N) if x.dim() == 1 else y


def hss_apply_raw(F: Factor, nrhs: int, x: torch.Tensor, y: torch.Tensor, ld: int, stream=None):
    """y = M^-1 x on column-major storage already laid out (no copies)."""
    _check(_lib.hss_apply(F.h, nrhs, _ptr(x), ld, _ptr(y), ld, _stream(stream)))


def hss_spmv(A: DeviceBSR, x: torch.Tensor, stream=None) -> torch.Tensor:
    N = A.n
    xs, k = _colmajor(x, N)
    ys = torch.empty_like(xs)
    _check(_lib.hss_spmv(C.byref(A.c), k, _ptr(xs), N, _ptr(ys), N, _stream(stream)))
    y = ys.t()
    return y.reshape(N) if x.dim() == 1 else y


@dataclass
class SolveStats:
    iters: int
    max_iters: int
    relres: float
    converged: bool


class ILU0:
    """Block ILU(0) of a device BSR matrix (the comparison preconditioner)."""

    def __init__(self, handle, A):
        self.h = C.c_void_p(handle)
        self.A = A                # keeps the matrix alive
        self.ndof = A.n

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ilu0_destroy(self.h)
            self.h = None


def ilu0_factor(A: DeviceBSR, stream=None) -> ILU0:
    out = C.c_void_p()
    _check(_lib.ilu0_factor(C.byref(A.c), _stream(stream), C.byref(out)))
    return ILU0(out.value, A)


def ilu0_apply(M: ILU0, x: torch.Tensor, stream=None) -> torch.Tensor:
    N = M.ndof
    xs, k = _colmajor(x, N)
    ys = torch.empty_like(xs)
    _check(_lib.ilu0_apply(M.h, k, _ptr(xs), N, _ptr(ys), N, _stream(stream)))
    y = ys.t()
    return y.reshape(N) if x.dim() == 1 else y


def fgmres_solve(A: DeviceBSR, F, b: torch.Tensor, x0: torch.Tensor | None = None,
                 restart=30, rtol=1e-8, maxit=1000, stream=None):
    """F: a Factor (the HSS preconditioner), an ILU0, or None (no preconditioner)."""
    N = A.n
    bs_, k = _colmajor(b, N)
    xs = torch.zeros_like(bs_) if x0 is None else _colmajor(x0, N)[0]
    o = fgmres_opts(restart, rtol, maxit)
    st = fgmres_stats()
    if isinstance(F, ILU0):
        _check(_lib.fgmres_solve_ilu0(C.byref(A.c), F.h, k, _ptr(bs_), N, _ptr(xs), N, C.byref(o), C.byref(st),
                                      _stream(stream)), allow=(HSS_ENOCONV,))
    else:
        _check(_lib.fgmres_solve(C.byref(A.c), F.h if F is not None else None, k, _ptr(bs_), N, _ptr(xs), N,
                                 C.byref(o), C.byref(st), _stream(stream)), allow=(HSS_ENOCONV,))
    x = xs.t()
    return (x.reshape(N) if b.dim() == 1 else x), SolveStats(st.iters, st.max_iters, st.relres, bool(st.converged))


def _mesh_struct(mesh):
    dim, n, p = mesh
    n3 = list(n) + [1] * (3 - len(n))
    return hss_mesh(dim, (C.c_int * 3)(*n3), p)


def nd_order_batched(meshes, As, leaf_max=64, scheme="box", stream=None) -> Tree:
    """Forest of independent instances (same block size).  The returned tree
    carries `inst_dof`: the first forest dof of each instance (ninst + 1)."""
    k = len(meshes)
    assert k == len(As) and k >= 1
    ms = (hss_mesh * k)(*[_mesh_struct(m) for m in meshes])
    bs = (hss_bsr * k)(*[A.c for A in As])
    o = hss_nd_opts(leaf_max, SCHEMES[scheme])
    out = C.c_void_p()
    _check(_lib.nd_order_batched(k, ms, bs, C.byref(o), _stream(stream), C.byref(out)))
    t = Tree(out.value, list(meshes))
    t.ninst = k
    t.inst_dof = np.concatenate([[0], np.cumsum([A.n for A in As])]).astype(np.int64)
    return t


def hss_factor_batched(As, forest: Tree, stream=None, **kw) -> Factor:
    o = factor_opts(**kw)
    k = len(As)
    bs = (hss_bsr * k)(*[A.c for A in As])
    out = C.c_void_p()
    _check(_lib.hss_factor_batched(k, bs, forest.h, C.byref(o), _stream(stream), C.byref(out)))
    return Factor(out.value, forest, o.precision)


def fgmres_solve_batched(F: Factor, B: torch.Tensor, x0: torch.Tensor | None = None, restart=30, rtol=1e-8,
                         maxit=1000, stream=None):
    """B: forest right-hand sides (ndof,) or (ndof, nrhs).  Returns X and one
    SolveStats per instance."""
    N = F.tree.desc.ndof
    bs_, k = _colmajor(B, N)
    xs = torch.zeros_like(bs_) if x0 is None else _colmajor(x0, N)[0]
    o = fgmres_opts(restart, rtol, maxit)
    ninst = F.tree.ninst
    st = (fgmres_stats * ninst)()
    _check(_lib.fgmres_solve_batched(F.h, k, _ptr(bs_), N, _ptr(xs), N, C.byref(o), st, _stream(stream)),
           allow=(HSS_ENOCONV,))
    x = xs.t()
    stats = [SolveStats(s_.iters, s_.max_iters, s_.relres, bool(s_.converged)) for s_ in st]
    return (x.reshape(N) if B.dim() == 1 else x), stats


RANK_NPARAMS = 8833


def rank_features(tree: Tree, c_elem=None, kappa_h=0.0) -> np.ndarray:
    """(nbox, 6) float32 features of every box (HOST)."""
    out = np.zeros((tree.desc.nbox, 6), dtype=np.float32)
    c = None if c_elem is None else np.ascontiguousarray(c_elem, dtype=np.float64)
    _check(_lib.hss_rank_features(tree.h, None if c is None else c.ctypes.data, float(kappa_h), out.ctypes.data))
    return out


class RankModel:
    """MLP predicting each front's largest HSS rank (FP32 training kernels,
    BF16 inference kernel)."""

    def __init__(self, seed=0):
        out = C.c_void_p()
        _check(_lib.hss_rank_model_create(seed, C.byref(out)))
        self.h = out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hss_rank_model_destroy(self.h)
            self.h = None

    def get(self):
        th = np.zeros(RANK_NPARAMS, dtype=np.float32)
        nm = np.zeros(14, dtype=np.float32)
        _check(_lib.hss_rank_model_get(self.h, th.ctypes.data, nm.ctypes.data))
        return th, nm

    def set(self, params=None, norm=None):
        th = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        nm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _check(_lib.hss_rank_model_set(self.h, None if th is None else th.ctypes.data,
                                       None if nm is None else nm.ctypes.data))

    @staticmethod
    def _dev(feat, target=None):
        f = torch.as_tensor(np.ascontiguousarray(feat, dtype=np.float32), device="cuda").contiguous()
        t = None if target is None else torch.as_tensor(np.ascontiguousarray(target, dtype=np.float32),
                                                        device="cuda").contiguous()
        return f, t

    def fit_norm(self, feat, target, stream=None):
        f, t = self._dev(feat, target)
        _check(_lib.hss_rank_model_fit_norm(self.h, f.shape[0], _ptr(f), _ptr(t), _stream(stream)))

    def loss_grad(self, feat, target, stream=None):
        f, t = self._dev(feat, target)
        loss = C.c_float()
        g = np.zeros(RANK_NPARAMS, dtype=np.float32)
        _check(_lib.hss_rank_model_loss_grad(self.h, f.shape[0], _ptr(f), _ptr(t), C.byref(loss), g.ctypes.data,
                                             _stream(stream)))
        return loss.value, g

    def train(self, feat, target, epochs=200, batch=256, lr=1e-3, seed=0, stream=None):
        f, t = self._dev(feat, target)
        loss = C.c_float()
        _check(_lib.hss_rank_model_train(self.h, f.shape[0], _ptr(f), _ptr(t), epochs, batch, lr, seed,
                                         C.byref(loss), _stream(stream)))
        return loss.value

    def predict(self, feat, oversample=10, rmax=96, stream=None):
        f, _ = self._dev(feat)
        n = f.shape[0]
        pred = torch.empty(n, dtype=torch.float32, device="cuda")
        r = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(_lib.hss_rank_model_predict(self.h, n, _ptr(f), oversample, rmax, _ptr(pred), _ptr(r),
                                           _stream(stream)))
        return pred.cpu().numpy(), r.cpu().numpy()


def fgmres_history(rhs=0, cap=100000) -> np.ndarray:
    h = np.zeros(cap)
    n = _lib.fgmres_history(rhs, h.ctypes.data_as(C.POINTER(C.c_double)), cap)
    return h[:n]


def launch_count() -> int:
    return int(_lib.hss_launch_count())


def gemm_tuner_choices() -> list:
    """The GEMM engine tuner's choices so far: dicts with the shape class
    (log2 of m, n, k rounded up, transposed A, generated B, tensor-core kernel
    timed), the engine kept and both times in ms."""
    n = _lib.hss_gemm_tuner_read(-1, None, None, None, None)
    out = []
    for i in range(n):
        key, eng, t0, t1 = C.c_longlong(), C.c_int(), C.c_float(), C.c_float()
        _check(_lib.hss_gemm_tuner_read(i, C.byref(key), C.byref(eng), C.byref(t0), C.byref(t1)))
        k = key.value
        out.append(dict(log2_m=(k >> 24) & 0xFFF, log2_n=(k >> 12) & 0xFFF, log2_k=k & 0xFFF,
                        trans_a=bool((k >> 39) & 1), gen_b=bool((k >> 38) & 1),
                        tc_kernel={1: "tma", 2: "staged"}.get((k >> 40) & 0xFF, "?"),
                        engine="simt" if eng.value == 0 else "tc", ms_simt=t0.value, ms_tc=t1.value))
    return out


def alloc_count() -> int:
    """Memory requests the library has served so far (hss_alloc_count)."""
    return int(_lib.hss_alloc_count())


def tc_timeout_selftest(spin_limit: int = 1 << 12, stream=None) -> int:
    """Runs the tensor-core kernel with its MMAs left out so that its bounded
    wait expires; returns the library's code (HSS_ETIMEOUT expected)."""
    return int(_lib.hss_tc_timeout_selftest(spin_limit, _stream(stream)))


def profile_enable(on: bool = True, host_only: bool = False):
    """Per-kernel-class event timing plus host-section timing; host_only
    records the host sections alone (no events)."""
    _check(_lib.hss_profile_enable((2 if host_only else 1) if on else 0))


def profile_reset():
    _check(_lib.hss_profile_reset())


def _profile_classes() -> dict:
    n = _lib.hss_profile_read(-1, None, 0, None, None, None)
    out = {}
    for i in range(n):
        name = C.create_string_buffer(64)
        ms, cnt, work = C.c_double(), C.c_long(), C.c_double()
        _check(_lib.hss_profile_read(i, name, 64, C.byref(ms), C.byref(cnt), C.byref(work)))
        out[name.value.decode()] = (ms.value, cnt.value, work.value)
    return out


def profile_read() -> dict:
    """{kernel class: (total_ms, launches, work)} of the events recorded so far."""
    return {k: v for k, v in _profile_classes().items() if not k.startswith("host:")}


def profile_read_host() -> dict:
    """{host section: (total host ms, entries)} recorded so far."""
    return {k[5:]: (v[0], v[1]) for k, v in _profile_classes().items() if k.startswith("host:")}


def gemm_f32(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, alpha=1.0, beta=0.0, engine=1,
             stream=None) -> torch.Tensor:
    """C = alpha A B + beta C on FP32 CUDA tensors (row-major torch tensors are
    handled as their column-major transposes: C^t = B^t A^t)."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if C is None:
        C = torch.zeros(m, n, dtype=torch.float32, device=A.device)
    At, Bt, Ct = A.contiguous(), B.contiguous(), C
    assert Ct.is_contiguous()
    # row-major (m x n) C is column-major (n x m) C^t = B^t A^t
    _check(_lib.hss_gemm_f32(n, m, k, _ptr(Bt), n, _ptr(At), max(k, 1), _ptr(Ct), n, alpha, beta, engine,
                             _stream(stream)))
    return Ct


GEMM_STATIC_MAX_TILES = 16384


def gemm_f32_static(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, alpha=1.0, beta=0.0, engine=1,
                    stream=None) -> torch.Tensor:
    """gemm_f32 through hss_gemm_f32_static (launch records in the library's
    fixed device array, no allocation in the call).  C must be given: this
    wrapper allocates nothing either."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2 and C.shape == (m, n)
    assert A.is_contiguous() and B.is_contiguous() and C.is_contiguous()
    _check(_lib.hss_gemm_f32_static(n, m, k, _ptr(B), n, _ptr(A), max(k, 1), _ptr(C), n, alpha, beta, engine,
                                    _stream(stream)))
    return C
