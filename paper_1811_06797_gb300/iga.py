"""ctypes binding of libiga (argument marshalling only).

Every function here forwards to the C entry point of the same name in
``libiga.so`` (declared in include/iga.h).  Device buffers are torch CUDA
tensors passed by pointer; host arrays are numpy arrays.  There is no
fallback path: if the library is missing or a call fails, an exception is
raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libiga.so")
_lib = None

IGA_FP64, IGA_FP32, IGA_TF32, IGA_BF16 = 0, 1, 2, 3
IGA_TRUNC_PIVOTED, IGA_TRUNC_SVD = 0, 1
IGA_RESID_FULL, IGA_RESID_LOCAL = 0, 1
STATUS = {0: "IGA_OK", 1: "IGA_EINVAL", 2: "IGA_ENOMEM", 3: "IGA_ECUDA", 4: "IGA_ENOCONV",
          5: "IGA_ENONFINITE", 6: "IGA_ETIMEOUT"}


class IgaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry_(C.Structure):
    _fields_ = [("kind", C.c_int), ("degree", C.c_int * 3), ("nknots", C.c_int * 3),
                ("knots", C.POINTER(C.c_double) * 3), ("nctrl", C.c_int * 3),
                ("ctrl_hw", C.POINTER(C.c_double)), ("twist", C.c_double)]


class Space_(C.Structure):
    _fields_ = [("degree", C.c_int * 3), ("nknots", C.c_int * 3),
                ("knots", C.POINTER(C.c_double) * 3), ("nquad", C.c_int)]


class Target_(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 4)]


class SolveOpts_(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("max_sweeps", C.c_int),
                ("kick_rank", C.c_int), ("rmax", C.c_int), ("local_maxit", C.c_int),
                ("refine_max", C.c_int), ("precision", C.c_int), ("verbose", C.c_int),
                ("trunc_tol", C.c_double), ("truncation", C.c_int), ("residual", C.c_int),
                ("state_weight", C.c_double)]


class SolveInfo_(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("refinements", C.c_int), ("max_rank", C.c_int),
                ("local_iters", C.c_int), ("residual", C.c_double), ("seconds", C.c_double),
                ("t_local", C.c_double), ("t_residual", C.c_double), ("t_move", C.c_double),
                ("t_refine", C.c_double)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libiga.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise IgaError(1, f"libiga.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(_LIB_PATH)
    vp, i, d, st = C.c_void_p, C.c_int, C.c_double, C.c_int
    P = C.POINTER
    sig = {
        "iga_create": (st, [P(vp), vp]),
        "iga_destroy": (None, [vp]),
        "iga_last_error": (C.c_char_p, [vp]),
        "iga_launch_count": (C.c_uint64, [vp]),
        "iga_scratch_bytes": (C.c_size_t, [vp]),
        "iga_profile_begin": (st, [vp, C.c_char_p]),
        "iga_profile_end": (st, [vp, P(C.c_uint64), P(d), P(d), P(d)]),
        "iga_measure_fma": (st, [vp, i, P(d)]),
        "iga_kkt_residual_rows": (st, [vp, vp, vp, d, vp, vp, vp, vp, i, P(C.c_int), P(d)]),
        "iga_gemm_batched": (st, [vp, i, i, i, i, i, i, d, vp, i, C.c_longlong, vp, i,
                                  C.c_longlong, d, vp, i, C.c_longlong, i]),
        "iga_sample_weights": (st, [vp, P(Geometry_), P(Space_), P(Target_), vp]),
        "iga_tt_svd": (st, [vp, vp, i, i, i, d, d, i, P(vp)]),
        "iga_tt_info": (st, [vp, P(C.c_int), P(C.c_int)]),
        "iga_tt_core": (st, [vp, vp, i, vp]),
        "iga_tt_full": (st, [vp, vp, vp]),
        "iga_tt_destroy": (None, [vp]),
        "iga_tt_save": (st, [vp, vp, C.c_char_p]),
        "iga_tt_load": (st, [vp, C.c_char_p, P(vp)]),
        "iga_assemble_bands": (st, [vp, P(Space_), i, vp, i, i, i, i, vp]),
        "iga_lowrank_assemble": (st, [vp, P(Geometry_), P(Space_), P(Target_), d, P(vp), P(vp),
                                      P(vp)]),
        "iga_weight_tts": (st, [vp, P(Geometry_), P(Space_), P(Target_), d, P(vp)]),
        "iga_lowrank_assemble_interp": (st, [vp, P(Geometry_), P(Space_), P(Target_), d, i,
                                             P(vp), P(vp), P(vp)]),
        "iga_weight_tts_interp": (st, [vp, P(Geometry_), P(Space_), P(Target_), d, i, P(vp)]),
        "iga_tt_from_cores": (st, [vp, P(C.c_int), P(C.c_int), P(vp), P(vp)]),
        "iga_ops_from_weights": (st, [vp, P(Space_), P(vp), P(vp), P(vp)]),
        "iga_load_from_density": (st, [vp, P(Space_), vp, P(vp)]),
        "iga_spd_solve": (st, [vp, vp, vp, vp, vp, vp, d, i, P(C.c_int), P(d)]),
        "iga_reduced_gradient": (st, [vp, vp, vp, vp, d, i, vp, d, vp, vp, vp, P(d)]),
        "iga_weight_gradient": (st, [vp, P(Space_), vp, vp, d, vp, vp, vp, vp]),
        "iga_op_from_bands": (st, [vp, P(C.c_int), P(C.c_int), i, P(C.c_int), P(vp), P(vp)]),
        "iga_op_info": (st, [vp, P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_int),
                             P(C.c_size_t)]),
        "iga_op_block": (st, [vp, i, P(C.c_int)]),
        "iga_op_bands": (st, [vp, vp, i, i, vp]),
        "iga_op_destroy": (None, [vp]),
        "iga_kron_apply": (st, [vp, vp, i, d, vp, d, vp, i]),
        "iga_kkt_apply": (st, [vp, vp, vp, d, vp, vp, i]),
        "iga_amen_local_matvec": (st, [vp, i, i, i, i, i, i, vp, vp, vp, vp, i, vp, vp, i]),
        "iga_amen_local_matvec_noalloc": (st, [vp, i, i, i, i, i, i, vp, vp, vp, vp, i, vp, vp,
                                               i]),
        "iga_solve_opts_default": (None, [P(SolveOpts_)]),
        "iga_kkt_solve_amen": (st, [vp, vp, vp, vp, d, P(SolveOpts_), vp, vp, vp,
                                    P(SolveInfo_)]),
        "iga_kkt_solve_amen_tt": (st, [vp, vp, vp, vp, d, P(SolveOpts_), P(vp), P(vp), P(vp),
                                       P(SolveInfo_)]),
        "iga_kkt_solve_parabolic": (st, [vp, vp, vp, i, d, vp, d, P(SolveOpts_), vp, vp, vp,
                                         P(SolveInfo_)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points this binding expects."""
    import re
    hdr = open(os.path.join(os.path.dirname(_HERE), "include", "iga.h")).read()
    return sorted(set(re.findall(r"\b(iga_[a-z0-9_]+)\s*\(", hdr)))


def _check(ctx, status):
    if status != 0:
        msg = lib().iga_last_error(ctx.handle if ctx is not None else None)
        raise IgaError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a contiguous torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise IgaError(1, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise IgaError(1, "expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return IGA_FP64
    if t.dtype == torch.float32:
        return IGA_FP32
    raise IgaError(1, f"unsupported dtype {t.dtype}")


class Context:
    """An iga_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = lib().iga_create(C.byref(h), C.c_void_p(stream.cuda_stream))
        if st != 0:
            raise IgaError(st, "iga_create failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().iga_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(lib().iga_launch_count(self.handle))

    @property
    def scratch_bytes(self) -> int:
        return int(lib().iga_scratch_bytes(self.handle))

    def last_error(self) -> str:
        return lib().iga_last_error(self.handle).decode()

    def profile_begin(self, kernel: str):
        _check(self, lib().iga_profile_begin(self.handle, kernel.encode()))

    def profile_end(self):
        n = C.c_uint64()
        ms, by, fl = C.c_double(), C.c_double(), C.c_double()
        _check(self, lib().iga_profile_end(self.handle, C.byref(n), C.byref(ms), C.byref(by),
                                          C.byref(fl)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}


def iga_measure_fma(ctx, prec):
    """Measured FMA rate of the CUDA cores in TFLOP/s (IGA_FP64 or IGA_FP32)."""
    r = C.c_double()
    _check(ctx, lib().iga_measure_fma(ctx.handle, int(prec), C.byref(r)))
    return r.value


def iga_gemm_batched(ctx, A, B, C, alpha=1.0, beta=0.0, tA=False, tB=False, tf32=False):
    """C[i] = alpha op(A[i]) op(B[i]) + beta C[i] for contiguous CUDA tensors
    of shape (count, rows, cols), all FP64 or all FP32, through the library's
    own dense product (tf32: FP32 tensors on the tensor cores)."""
    import torch
    for t in (A, B, C):
        if not (t.is_cuda and t.is_contiguous() and t.dim() == 3):
            raise IgaError(1, "gemm_batched: contiguous 3-d CUDA tensors expected")
        if t.dtype != A.dtype or t.device != A.device:
            raise IgaError(1, "gemm_batched: mixed dtypes or devices")
    if A.dtype not in (torch.float64, torch.float32):
        raise IgaError(1, "gemm_batched: FP64 or FP32 tensors expected")
    count = A.shape[0]
    M, K = (A.shape[2], A.shape[1]) if tA else (A.shape[1], A.shape[2])
    Kb, N = (B.shape[2], B.shape[1]) if tB else (B.shape[1], B.shape[2])
    if Kb != K or tuple(C.shape) != (count, M, N) or B.shape[0] != count:
        raise IgaError(1, "gemm_batched: shape mismatch")
    prec = IGA_FP64 if A.dtype == torch.float64 else IGA_FP32
    if tf32:
        if prec != IGA_FP32:
            raise IgaError(1, "gemm_batched: the TF32 path takes FP32 tensors")
        prec = IGA_TF32
    _check(ctx, lib().iga_gemm_batched(
        ctx.handle, prec, int(tA), int(tB), M, N, K, float(alpha), _ptr(A), A.shape[2],
        A.shape[1] * A.shape[2], _ptr(B), B.shape[2], B.shape[1] * B.shape[2], float(beta),
        _ptr(C), N, M * N, count))


class _Keep:
    """Holds host arrays alive while a C struct points into them."""

    def __init__(self):
        self.items = []

    def arr(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.items.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))


def geometry_struct(geo, keep):
    g = Geometry_()
    g.kind = int(geo.kind)
    for d in range(3):
        g.degree[d] = int(geo.degree[d])
        g.nknots[d] = len(geo.knots[d])
        g.knots[d] = keep.arr(geo.knots[d])
        g.nctrl[d] = int(geo.ctrl.shape[d])
    g.ctrl_hw = keep.arr(geo.homogeneous())
    g.twist = float(geo.twist)
    return g


def space_struct(space, keep):
    s = Space_()
    for d in range(3):
        s.degree[d] = int(space.degree[d])
        s.nknots[d] = len(space.knots[d])
        s.knots[d] = keep.arr(space.knots[d])
    s.nquad = int(space.nquad)
    return s


def target_struct(target):
    t = Target_()
    if target is None:
        t.kind = 0
        return t
    t.kind = int(target.kind)
    for k, v in enumerate(target.params()):
        t.params[k] = float(v)
    return t


class TT:
    """Library-owned TT tensor (iga_tt)."""

    def __init__(self, handle):
        self.handle = handle

    def info(self):
        n = (C.c_int * 3)()
        r = (C.c_int * 2)()
        _check(None, lib().iga_tt_info(self.handle, n, r))
        return tuple(n), tuple(r)

    def core(self, ctx, d):
        n, r = self.info()
        rl = (1, r[0], r[1], 1)
        out = np.empty((rl[d], n[d], rl[d + 1]))
        _check(ctx, lib().iga_tt_core(ctx.handle, self.handle, d, out.ctypes.data_as(C.c_void_p)))
        return out

    def cores(self, ctx):
        return [self.core(ctx, d) for d in range(3)]

    def full(self, ctx, out):
        _check(ctx, lib().iga_tt_full(ctx.handle, self.handle, _ptr(out)))
        return out

    def save(self, ctx, path):
        _check(ctx, lib().iga_tt_save(ctx.handle, self.handle, os.fsencode(path)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.iga_tt_destroy(self.handle)
            self.handle = None


class Op:
    """Library-owned Kronecker / TT-matrix operator (iga_op)."""

    def __init__(self, handle):
        self.handle = handle

    def info(self):
        n = (C.c_int * 3)()
        p = (C.c_int * 3)()
        nb = C.c_int()
        R = (C.c_int * 2)()
        by = C.c_size_t()
        _check(None, lib().iga_op_info(self.handle, n, p, C.byref(nb), R, C.byref(by)))
        return {"n": tuple(n), "p": tuple(p), "nblocks": nb.value, "R": tuple(R),
                "bytes": by.value}

    def block_ranks(self, k):
        R = (C.c_int * 2)()
        _check(None, lib().iga_op_block(self.handle, k, R))
        return tuple(R)

    def bands(self, ctx, k, d):
        inf = self.info()
        R1, R2 = self.block_ranks(k)
        b = 2 * inf["p"][d] + 1
        n = inf["n"][d]
        shape = {0: (R1, n, b), 1: (R1, R2, n, b), 2: (R2, n, b)}[d]
        out = np.empty(shape)
        _check(ctx, lib().iga_op_bands(ctx.handle, self.handle, k, d,
                                       out.ctypes.data_as(C.c_void_p)))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.iga_op_destroy(self.handle)
            self.handle = None


def iga_sample_weights(ctx, geometry, space, target, out):
    keep = _Keep()
    g = geometry_struct(geometry, keep)
    s = space_struct(space, keep)
    t = target_struct(target)
    _check(ctx, lib().iga_sample_weights(ctx.handle, C.byref(g), C.byref(s), C.byref(t), _ptr(out)))
    return out


def iga_tt_load(ctx, path):
    h = C.c_void_p()
    _check(ctx, lib().iga_tt_load(ctx.handle, os.fsencode(path), C.byref(h)))
    return TT(h)


def iga_tt_svd(ctx, W, tol, norm_ref=0.0, rmax=0):
    h = C.c_void_p()
    n1, n2, n3 = W.shape
    _check(ctx, lib().iga_tt_svd(ctx.handle, _ptr(W), n1, n2, n3, float(tol), float(norm_ref),
                                 int(rmax), C.byref(h)))
    return TT(h) if h.value else None


def iga_assemble_bands(ctx, space, d, w, deriv_row, deriv_col, interior, band):
    keep = _Keep()
    s = space_struct(space, keep)
    T = w.shape[0]
    _check(ctx, lib().iga_assemble_bands(ctx.handle, C.byref(s), d, _ptr(w), T, int(deriv_row),
                                         int(deriv_col), int(interior), _ptr(band)))
    return band


def iga_lowrank_assemble(ctx, geometry, space, target, tol):
    keep = _Keep()
    g = geometry_struct(geometry, keep)
    s = space_struct(space, keep)
    t = target_struct(target)
    hm, hk, hl = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(ctx, lib().iga_lowrank_assemble(ctx.handle, C.byref(g), C.byref(s), C.byref(t),
                                           float(tol), C.byref(hm), C.byref(hk), C.byref(hl)))
    return Op(hm), Op(hk), (TT(hl) if hl.value else None)


def iga_lowrank_assemble_interp(ctx, geometry, space, target, tol, degree=0):
    """Low-rank assembly with the weights interpolated in a spline space of the
    given degree (0: 2p + 1)."""
    keep = _Keep()
    g = geometry_struct(geometry, keep)
    s = space_struct(space, keep)
    t = target_struct(target)
    hm, hk, hl = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(ctx, lib().iga_lowrank_assemble_interp(ctx.handle, C.byref(g), C.byref(s), C.byref(t),
                                                  float(tol), int(degree), C.byref(hm),
                                                  C.byref(hk), C.byref(hl)))
    return Op(hm), Op(hk), (TT(hl) if hl.value else None)


def iga_weight_tts_interp(ctx, geometry, space, target, tol, degree=0):
    keep = _Keep()
    g = geometry_struct(geometry, keep)
    s = space_struct(space, keep)
    t = target_struct(target)
    hs = (C.c_void_p * 8)()
    _check(ctx, lib().iga_weight_tts_interp(ctx.handle, C.byref(g), C.byref(s), C.byref(t),
                                            float(tol), int(degree), hs))
    return [TT(C.c_void_p(h)) if h else None for h in hs]


def iga_weight_tts(ctx, geometry, space, target, tol):
    """The 8 sampled weight TTs (omega, q11, q12, q13, q22, q23, q33, load density)."""
    keep = _Keep()
    g = geometry_struct(geometry, keep)
    s = space_struct(space, keep)
    t = target_struct(target)
    hs = (C.c_void_p * 8)()
    _check(ctx, lib().iga_weight_tts(ctx.handle, C.byref(g), C.byref(s), C.byref(t), float(tol),
                                     hs))
    return [TT(C.c_void_p(h)) if h else None for h in hs]


def iga_tt_from_cores(ctx, cores):
    """TT from three device core tensors (1,n1,r1), (r1,n2,r2), (r2,n3,1)."""
    n = (C.c_int * 3)(*[c.shape[1] for c in cores])
    r = (C.c_int * 2)(cores[0].shape[2], cores[1].shape[2])
    ptrs = (C.c_void_p * 3)(*[c.data_ptr() for c in cores])
    for c in cores:
        _ptr(c)
    h = C.c_void_p()
    _check(ctx, lib().iga_tt_from_cores(ctx.handle, n, r, ptrs, C.byref(h)))
    return TT(h)


def iga_ops_from_weights(ctx, space, weights):
    """M, K from 7 weight TTs (omega, q11, q12, q13, q22, q23, q33; None = zero)."""
    keep = _Keep()
    s = space_struct(space, keep)
    hs = (C.c_void_p * 7)(*[(w.handle.value if w is not None else None) for w in weights])
    hm, hk = C.c_void_p(), C.c_void_p()
    _check(ctx, lib().iga_ops_from_weights(ctx.handle, C.byref(s), hs, C.byref(hm), C.byref(hk)))
    return Op(hm), Op(hk)


def iga_op_from_bands(ctx, blocks):
    """Operator from banded factors: blocks = [(A1, A2, A3), ...] FP64 CUDA
    tensors of shapes (R1, n1, 2p+1), (R1, R2, n2, 2p+1), (R2, n3, 2p+1)."""
    nb = len(blocks)
    if nb == 0:
        raise IgaError(1, "no blocks")
    A1, A2, A3 = blocks[0]
    n = (C.c_int * 3)(A1.shape[1], A2.shape[2], A3.shape[1])
    p = (C.c_int * 3)(*[(t.shape[-1] - 1) // 2 for t in (A1, A2, A3)])
    R = (C.c_int * (2 * nb))()
    ptrs = (C.c_void_p * (3 * nb))()
    for k, (a1, a2, a3) in enumerate(blocks):
        R[2 * k], R[2 * k + 1] = a1.shape[0], a3.shape[0]
        if tuple(a2.shape[:2]) != (a1.shape[0], a3.shape[0]):
            raise IgaError(1, "A2 must be (R1, R2, n2, 2p+1)")
        for d, t in enumerate((a1, a2, a3)):
            ptrs[3 * k + d] = _ptr(t).value
            if t.dtype.itemsize != 8:
                raise IgaError(1, "bands must be float64")
    h = C.c_void_p()
    _check(ctx, lib().iga_op_from_bands(ctx.handle, n, p, nb, R, ptrs, C.byref(h)))
    return Op(h)


def iga_load_from_density(ctx, space, density):
    keep = _Keep()
    s = space_struct(space, keep)
    h = C.c_void_p()
    _check(ctx, lib().iga_load_from_density(ctx.handle, C.byref(s), density.handle, C.byref(h)))
    return TT(h)


def iga_spd_solve(ctx, A, M, K, b, x, tol=1e-12, maxit=2000):
    it = C.c_int()
    rr = C.c_double()
    _check(ctx, lib().iga_spd_solve(ctx.handle, A.handle, M.handle,
                                    K.handle if K is not None else None, _ptr(b), _ptr(x),
                                    float(tol), int(maxit), C.byref(it), C.byref(rr)))
    return {"iters": it.value, "relres": rr.value}


def iga_reduced_gradient(ctx, M, K, load, beta, u, grad, y, lam, tol=1e-12):
    """u, grad, y, lam: (nbatch, N) or (N,) FP64 device tensors; returns J per control."""
    nbatch = 1 if u.dim() == 1 else u.shape[0]
    J = (C.c_double * nbatch)()
    _check(ctx, lib().iga_reduced_gradient(ctx.handle, M.handle, K.handle,
                                           load.handle if load is not None else None,
                                           float(beta), nbatch, _ptr(u), float(tol), _ptr(grad),
                                           _ptr(y), _ptr(lam), J))
    return np.array(J[:])


def iga_weight_gradient(ctx, space, M, K, beta, y, u, lam, grad_w):
    keep = _Keep()
    s = space_struct(space, keep)
    _check(ctx, lib().iga_weight_gradient(ctx.handle, C.byref(s), M.handle, K.handle, float(beta),
                                          _ptr(y), _ptr(u), _ptr(lam), _ptr(grad_w)))
    return grad_w


def iga_kron_apply(ctx, A, alpha, x, beta, y, tf32=False, bf16=False, transpose=False):
    """y = alpha op(A) x + beta y (op(A) = A^T with transpose=True); float32
    tensors with tf32=True (bf16=True) run the rank contraction of TT-matrix
    blocks on the tensor cores with TF32 (BF16) operands."""
    if x.dtype != y.dtype:
        raise IgaError(1, "x and y dtypes differ")
    prec = _prec(x)
    if tf32 or bf16:
        if prec != IGA_FP32 or (tf32 and bf16):
            raise IgaError(1, "tf32 / bf16 need float32 tensors (one of the two)")
        prec = IGA_TF32 if tf32 else IGA_BF16
    _check(ctx, lib().iga_kron_apply(ctx.handle, A.handle, int(bool(transpose)), float(alpha),
                                     _ptr(x), float(beta), _ptr(y), prec))
    return y


def iga_kkt_apply(ctx, M, K, beta, z, out):
    if z.dtype != out.dtype:
        raise IgaError(1, "z and out dtypes differ")
    _check(ctx, lib().iga_kkt_apply(ctx.handle, M.handle, K.handle, float(beta), _ptr(z),
                                    _ptr(out), _prec(z)))
    return out


def _local_matvec_args(PhiL, bands, PhiR, x, y, bandmask):
    """Check the operands of a local matvec before any launch.

    All five tensors must be contiguous CUDA tensors of one dtype (float64 or
    float32) on one device, with PhiL (R0, r0, r0), bands (R0, R1, n, 2p+1),
    PhiR (R1, r1, r1) and x, y (nvec, r0, n, r1); a band mask has R0 * R1
    entries.  Returns the sizes and the host mask pointer (or None).
    """
    ts = {"PhiL": PhiL, "bands": bands, "PhiR": PhiR, "x": x, "y": y}
    for name, t in ts.items():
        if t is None or not t.is_cuda:
            raise IgaError(1, f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise IgaError(1, f"{name} must be contiguous")
        if t.dtype != x.dtype:
            raise IgaError(1, f"{name} has dtype {t.dtype}, x has {x.dtype}")
        if t.device != x.device:
            raise IgaError(1, f"{name} is on {t.device}, x is on {x.device}")
    _prec(x)
    if PhiL.dim() != 3 or PhiR.dim() != 3 or bands.dim() != 4 or x.dim() != 4:
        raise IgaError(1, "expected PhiL (R0,r0,r0), bands (R0,R1,n,2p+1), PhiR (R1,r1,r1), "
                          "x (nvec,r0,n,r1)")
    R0, r0, r0b = PhiL.shape
    R1, r1, r1b = PhiR.shape
    nvec, xr0, n, xr1 = x.shape
    if r0b != r0 or r1b != r1:
        raise IgaError(1, "PhiL and PhiR must be square in their last two dimensions")
    if tuple(bands.shape[:3]) != (R0, R1, n) or bands.shape[3] % 2 != 1:
        raise IgaError(1, f"bands must be ({R0}, {R1}, {n}, 2p+1), got {tuple(bands.shape)}")
    if (xr0, xr1) != (r0, r1) or tuple(y.shape) != tuple(x.shape):
        raise IgaError(1, f"x and y must be (nvec, {r0}, {n}, {r1})")
    if x.data_ptr() == y.data_ptr():
        raise IgaError(1, "x and y must not overlap")
    mask = keep = None
    if bandmask is not None:
        keep = np.ascontiguousarray(bandmask, dtype=np.uint8)
        if keep.size != R0 * R1:
            raise IgaError(1, f"bandmask must have R0 * R1 = {R0 * R1} entries")
        mask = keep.ctypes.data_as(C.POINTER(C.c_ubyte))
    p = (bands.shape[3] - 1) // 2
    return (r0, n, r1, R0, R1, p, nvec), mask, keep


def iga_amen_local_matvec(ctx, PhiL, bands, PhiR, x, y, bandmask=None):
    """PhiL (R0,r0,r0), bands (R0,R1,n,2p+1), PhiR (R1,r1,r1), x/y (nvec,r0,n,r1)."""
    (r0, n, r1, R0, R1, p, nvec), mask, keep = _local_matvec_args(PhiL, bands, PhiR, x, y,
                                                                  bandmask)
    _check(ctx, lib().iga_amen_local_matvec(ctx.handle, r0, n, r1, R0, R1, p, _ptr(PhiL),
                                            _ptr(bands), _ptr(PhiR), mask, nvec, _ptr(x),
                                            _ptr(y), _prec(x)))
    del keep
    return y


def iga_amen_local_matvec_noalloc(PhiL, bands, PhiR, x, y, bandmask=None, stream=None):
    """Allocation-free local matvec on `stream` (default: the current stream of x's device).

    Same contraction as iga_amen_local_matvec, using the library's fixed
    device scratch instead of allocating; raises IgaError (IGA_EINVAL) for
    sizes beyond that fixed scratch.  The call runs with x's device current,
    so the library picks that device's scratch.
    """
    import torch
    (r0, n, r1, R0, R1, p, nvec), mask, keep = _local_matvec_args(PhiL, bands, PhiR, x, y,
                                                                  bandmask)
    with torch.cuda.device(x.device):
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        if s.device != x.device:
            raise IgaError(1, f"stream is on {s.device}, the tensors on {x.device}")
        st = lib().iga_amen_local_matvec_noalloc(C.c_void_p(s.cuda_stream), r0, n, r1, R0, R1,
                                                 p, _ptr(PhiL), _ptr(bands), _ptr(PhiR), mask,
                                                 nvec, _ptr(x), _ptr(y), _prec(x))
    del keep
    if st != 0:
        raise IgaError(st, "iga_amen_local_matvec_noalloc failed (sizes beyond the fixed "
                           "16 MiB scratch, invalid arguments or a CUDA error)")
    return y


def solve_opts(**kw):
    o = SolveOpts_()
    lib().iga_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise IgaError(1, f"unknown solve option {k}")
        setattr(o, k, v)
    return o


def iga_kkt_solve_amen(ctx, M, K, load, beta, y, u, lam, **opts):
    o = solve_opts(**opts)
    info = SolveInfo_()
    st = lib().iga_kkt_solve_amen(ctx.handle, M.handle, K.handle,
                                  load.handle if load is not None else None, float(beta),
                                  C.byref(o), _ptr(y), _ptr(u), _ptr(lam), C.byref(info))
    res = {f: getattr(info, f) for f, _ in SolveInfo_._fields_}
    if st not in (0, 4):
        _check(ctx, st)
    res["converged"] = st == 0
    return res


def iga_kkt_residual_rows(ctx, M, K, beta, load, y, u, lam, rows):
    """Residuals of the three KKT equations at the interior multi-indices
    `rows` ((S, 3) integers, 0-based) for a solution given as TT handles:
    a numpy array (S, 3)."""
    import numpy as np
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((r.shape[0], 3), dtype=np.float64)
    _check(ctx, lib().iga_kkt_residual_rows(
        ctx.handle, M.handle, K.handle, float(beta), load.handle if load is not None else None,
        y.handle, u.handle, lam.handle, r.shape[0],
        r.ctypes.data_as(C.POINTER(C.c_int)), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def iga_kkt_solve_parabolic(ctx, M, K, nt, tau, load, beta, y, u, lam, **opts):
    """The parabolic KKT solve (nt implicit Euler steps of size tau): load,
    y, u, lam are float64 CUDA tensors of nt x N elements (time the slow
    index; load may be None).  Returns the solve info with `converged`."""
    import torch
    N = int(np.prod(M.info()["n"]))
    ts = [t for t in (load, y, u, lam) if t is not None]
    for t in ts:
        if t.dtype != torch.float64 or t.numel() != int(nt) * N:
            raise IgaError(1, "kkt_solve_parabolic: expected float64 tensors of nt * N elements")
        if t.device != y.device:
            raise IgaError(1, "kkt_solve_parabolic: tensors on different devices")
    o = solve_opts(**opts)
    info = SolveInfo_()
    with torch.cuda.device(y.device):
        st = lib().iga_kkt_solve_parabolic(ctx.handle, M.handle, K.handle, int(nt), float(tau),
                                           _ptr(load), float(beta), C.byref(o), _ptr(y), _ptr(u),
                                           _ptr(lam), C.byref(info))
    res = {f: getattr(info, f) for f, _ in SolveInfo_._fields_}
    if st not in (0, 4):
        _check(ctx, st)
    res["converged"] = st == 0
    return res


def iga_kkt_solve_amen_tt(ctx, M, K, load, beta, **opts):
    """The KKT solve with the solution as TT handles: (y, u, lam, info)."""
    o = solve_opts(**opts)
    info = SolveInfo_()
    hs = [C.c_void_p() for _ in range(3)]
    st = lib().iga_kkt_solve_amen_tt(ctx.handle, M.handle, K.handle,
                                     load.handle if load is not None else None, float(beta),
                                     C.byref(o), C.byref(hs[0]), C.byref(hs[1]), C.byref(hs[2]),
                                     C.byref(info))
    res = {f: getattr(info, f) for f, _ in SolveInfo_._fields_}
    if st not in (0, 4):
        _check(ctx, st)
    res["converged"] = st == 0
    return tuple(TT(h) if h.value else None for h in hs) + (res,)
