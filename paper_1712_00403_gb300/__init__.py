"""GB300 (sm_103a) library for Fast-Diagonalization-preconditioned MINRES on
the isogeometric Stokes system (Montardini, Sangalli, Tani, arXiv 1712.00403).

Thin ctypes binding over the C ABI declared in include/fdst.h: argument
marshalling only, every step of the computation runs in the library's CUDA
kernels. PyTorch supplies device memory and streams. The compiled library
is loaded on first use (Stokes, Batch, Server and the module functions), which
raises ImportError when it is missing; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdst.so")

TH, RT = 0, 1
FD_F64, FD_TF32X3, FD_BF16X6 = 0, 1, 2
HAS_TC = True        # the split-TF32 tcgen05 FD contraction is built (sm_103a)
GEOM_IDENTITY, GEOM_SINE_BUMP, GEOM_ANNULUS = 0, 1, 2
VARIANT_PD, VARIANT_PD_GEO = 0, 1
MV_F64, MV_DF64 = 0, 1
MATVEC_ASSEMBLED, MATVEC_MATRIX_FREE = 0, 1
PREC_PT, PREC_PC = 0, 1
GMRES_LEFT, GMRES_FLEXIBLE, GMRES_AUTO = 0, 1, 2

STATUS = {0: "OK", 1: "INVALID_ARGUMENT", 2: "NOT_SPD", 3: "OUT_OF_MEMORY", 4: "CUDA_ERROR", 5: "MAXIT",
          6: "STAGNATION", 7: "BREAKDOWN", 8: "TIMEOUT", 9: "NAN_DETECTED", 10: "ADMISSION_REJECTED",
          11: "NOT_SUPPORTED", 12: "CANCELLED"}


BATCH_MODES = {0: "fp64", 1: "streamed", 2: "resident_b", 3: "resident_b_tmem_a"}


class FdstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("discretization", ctypes.c_int), ("degree", ctypes.c_int),
                ("h_knots", ctypes.POINTER(ctypes.c_double) * 3), ("nknots", ctypes.c_int * 3),
                ("viscosity", ctypes.c_double), ("geometry", ctypes.c_int), ("variant", ctypes.c_int),
                ("fd_precision", ctypes.c_int), ("cpen", ctypes.c_double), ("max_rhs", ctypes.c_int),
                ("matvec_precision", ctypes.c_int), ("geometry_amplitude", ctypes.c_double),
                ("viscosity_contrast", ctypes.c_double), ("matvec_form", ctypes.c_int)]


class Sizes(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_total", ctypes.c_int64), ("nblocks", ctypes.c_int),
                ("block_offset", ctypes.c_int64 * 4), ("block_shape", (ctypes.c_int * 3) * 4),
                ("device_bytes", ctypes.c_int64), ("flops_apply", ctypes.c_double),
                ("flops_matvec", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int), ("fd_precision", ctypes.c_int),
                ("matvec_precision", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("iters_per_step", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("eta_rel", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("iterations_estimate", ctypes.c_int)]


ENTRY_POINTS = ["fdst_setup", "fdst_destroy", "fdst_get_sizes", "fdst_apply_prec", "fdst_matvec", "fdst_solve",
                "fdst_solve_host", "fdst_solve_host_zero", "fdst_apply_prec_host", "fdst_solve_gmres", "fdst_apply_block_prec", "fdst_set_timing", "fdst_get_timing", "fdst_get_kernel_timing", "fdst_convert",
                "fdst_fd_apply_static", "fdst_batch_create", "fdst_batch_solve", "fdst_batch_info", "fdst_batch_tuning", "fdst_batch_set_tuning",
                "fdst_batch_destroy", "fdst_server_create", "fdst_server_submit", "fdst_server_step",
                "fdst_server_result", "fdst_server_stats", "fdst_server_cancel", "fdst_server_destroy",
                "fdst_check_bounded_wait", "fdst_device_error", "fdst_inject_alloc_failure",
                "fdst_kernel_launches", "fdst_last_error"]

_lib = None


def load_library(path=LIB_PATH):
    """Load libfdst.so (built by paper_1712_00403_gb300.build). Raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1712_00403_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.fdst_setup.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(vp)]
    lib.fdst_destroy.argtypes = [vp]
    lib.fdst_get_sizes.argtypes = [vp, ctypes.POINTER(Sizes)]
    lib.fdst_apply_prec.argtypes = [vp, vp, vp, i, vp]
    lib.fdst_matvec.argtypes = [vp, vp, vp, i, vp]
    lib.fdst_solve.argtypes = [vp, vp, vp, i, d, i, ctypes.POINTER(SolveInfo), vp]
    lib.fdst_solve_gmres.argtypes = [vp, i, i, vp, vp, i, d, i, i, ctypes.POINTER(SolveInfo), vp]
    lib.fdst_apply_block_prec.argtypes = [vp, i, vp, vp, i, vp]
    lib.fdst_check_bounded_wait.argtypes = [ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.fdst_solve_host.argtypes = [vp, vp, vp, i, d, i, ctypes.POINTER(SolveInfo), vp]
    lib.fdst_solve_host_zero.argtypes = [vp, vp, vp, i, d, i, ctypes.POINTER(SolveInfo), vp]
    lib.fdst_apply_prec_host.argtypes = [vp, vp, vp, i, vp]
    lib.fdst_set_timing.argtypes = [vp, i]
    lib.fdst_device_error.argtypes = [ctypes.POINTER(i)]
    lib.fdst_batch_create.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(vp)]
    lib.fdst_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), d, i, ctypes.POINTER(SolveInfo), vp]
    lib.fdst_batch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.fdst_batch_tuning.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fdst_batch_set_tuning.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fdst_batch_destroy.argtypes = [vp]
    lib.fdst_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.fdst_server_submit.argtypes = [vp, ctypes.POINTER(Desc), vp, d, ctypes.POINTER(i64)]
    lib.fdst_server_step.argtypes = [vp, d, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i64)]
    lib.fdst_server_result.argtypes = [vp, i64, ctypes.POINTER(i), vp, ctypes.POINTER(SolveInfo),
                                       ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.fdst_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64), ctypes.POINTER(i)]
    lib.fdst_server_destroy.argtypes = [vp]
    lib.fdst_server_cancel.argtypes = [vp, i64]
    lib.fdst_inject_alloc_failure.argtypes = [i64, i]
    lib.fdst_fd_apply_static.argtypes = [i, ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(d), vp, vp, vp]
    lib.fdst_get_timing.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                    ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.fdst_get_kernel_timing.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64)]
    lib.fdst_convert.argtypes = [i, vp, vp, ctypes.c_int64, vp]
    lib.fdst_last_error.restype = ctypes.c_char_p
    lib.fdst_last_error.argtypes = []
    for name in ENTRY_POINTS[:-2]:
        getattr(lib, name).restype = ctypes.c_int
    lib.fdst_kernel_launches.restype = ctypes.c_int64
    lib.fdst_kernel_launches.argtypes = []
    _lib = lib
    return lib


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load_library().fdst_kernel_launches())


def fd_apply_static(U, lam, coef, r, s, stream=None):
    """Allocation-free FD solve of one Kronecker-sum block (fdst_fd_apply_static).

    U, lam: lists (one per direction, 2 or 3) of CUDA float64 tensors holding
    U_d (n_d x n_d, row-major) and lam_d; coef: per-direction coefficients;
    r, s: CUDA float64 vectors of prod(n_d) entries (i1 fastest). For callers
    that cannot allocate device memory; see include/fdst.h for the scratch
    limits and the rule that overlapping calls race.

    The C entry point cannot see buffer lengths, so every size is checked
    here before the call: ValueError for a dimension outside {2, 3}, unequal
    list lengths, a non-square U_d, a lam_d, r or s of the wrong length;
    TypeError for a tensor that is not a contiguous float64 CUDA tensor.
    """
    dim = len(U)
    if dim not in (2, 3):
        raise ValueError(f"fd_apply_static: 2 or 3 directions, got {dim}")
    if len(lam) != dim or len(coef) != dim:
        raise ValueError(f"fd_apply_static: {dim} factors need {dim} eigenvalue vectors and {dim} coefficients, "
                         f"got {len(lam)} and {len(coef)}")
    n = []
    for d in range(dim):
        if U[d].dim() != 2 or U[d].shape[0] != U[d].shape[1]:
            raise ValueError(f"fd_apply_static: U_{d + 1} must be square, got shape {tuple(U[d].shape)}")
        n.append(int(U[d].shape[0]))
        if lam[d].numel() != n[d]:
            raise ValueError(f"fd_apply_static: lam_{d + 1} has {lam[d].numel()} entries, U_{d + 1} is {n[d]} x {n[d]}")
    N = 1
    for v in n:
        N *= v
    for name, t in (("r", r), ("s", s)):
        if t.numel() != N:
            raise ValueError(f"fd_apply_static: {name} has {t.numel()} entries, the block has {N}")
    ptrs = [_dptr(t).value for t in (*U, *lam, r, s)]
    lib = load_library()
    nn = (ctypes.c_int * 3)(*n, *([1] * (3 - dim)))
    up = (ctypes.c_void_p * 3)(*ptrs[:dim], *([None] * (3 - dim)))
    lp = (ctypes.c_void_p * 3)(*ptrs[dim:2 * dim], *([None] * (3 - dim)))
    cf = (ctypes.c_double * 3)(*[float(c) for c in coef], *([0.0] * (3 - dim)))
    _check(lib.fdst_fd_apply_static(dim, nn, up, lp, cf, ctypes.c_void_p(ptrs[-2]), ctypes.c_void_p(ptrs[-1]),
                                    _stream_ptr(stream)))


CONVERT_F64_TO_F32, CONVERT_F64_TO_DF, CONVERT_DF_TO_F64, CONVERT_F32_TO_F64 = 0, 1, 2, 3


def convert(kind, src, dst, stream=None):
    """Element-wise precision conversion on the device (fdst_convert): src and dst
    contiguous CUDA tensors; a double-float pair is two float32 entries."""
    import torch
    want = {CONVERT_F64_TO_F32: (torch.float64, torch.float32), CONVERT_F64_TO_DF: (torch.float64, torch.float32),
            CONVERT_DF_TO_F64: (torch.float32, torch.float64), CONVERT_F32_TO_F64: (torch.float32, torch.float64)}
    n = src.numel() if kind != CONVERT_DF_TO_F64 else src.numel() // 2
    m = n * 2 if kind == CONVERT_F64_TO_DF else n
    for t, dt, cnt in ((src, want[kind][0], src.numel()), (dst, want[kind][1], m)):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt and t.numel() >= cnt):
            raise TypeError("convert: expected contiguous CUDA tensors of the kind's dtypes and sizes")
    _check(load_library().fdst_convert(int(kind), ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                       n, _stream_ptr(stream)))


def check_bounded_wait():
    """Failure-detection self-test (fdst_check_bounded_wait): (status, gave_up,
    seconds); status is "TIMEOUT" when the wait expired as designed."""
    g, t = ctypes.c_int(), ctypes.c_double()
    code = load_library().fdst_check_bounded_wait(ctypes.byref(g), ctypes.byref(t))
    if code not in (0, 8):
        _check(code)
    return STATUS[code], bool(g.value), t.value


def inject_alloc_failure(nth, status=3):
    """Host-side fault injection (fdst_inject_alloc_failure): the nth device
    allocation of a handle from now on fails with status (3 OUT_OF_MEMORY or
    4 CUDA_ERROR) without touching the GPU; nth <= 0 disarms."""
    _check(load_library().fdst_inject_alloc_failure(int(nth), int(status)))


def device_error():
    """1 when a bounded device-side wait in a tensor-core kernel expired."""
    f = ctypes.c_int()
    _check(load_library().fdst_device_error(ctypes.byref(f)))
    return f.value


def _check(code):
    if code != 0:
        raise FdstError(code, _lib.fdst_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Stokes:
    """One Stokes problem on the device: spaces, FD factors, operator and MINRES workspace.

    knots: list (one per direction) of open pressure knot vectors on [0,1];
    p: pressure degree. See include/fdst.h for the meaning of every option.
    """

    def __init__(self, knots, p, disc=TH, viscosity=1.0, fd_precision=FD_F64, max_rhs=1,
                 geometry=GEOM_IDENTITY, variant=VARIANT_PD, cpen=0.0, matvec_precision=MV_F64,
                 matvec_form=MATVEC_ASSEMBLED, geometry_amplitude=0.0, viscosity_contrast=0.0):
        lib = load_library()
        self._knots = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        desc = Desc()
        desc.dim = len(knots)
        desc.discretization = disc
        desc.degree = p
        for e, k in enumerate(self._knots):
            desc.h_knots[e] = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            desc.nknots[e] = len(k)
        desc.viscosity = viscosity
        desc.geometry = geometry
        desc.variant = variant
        desc.fd_precision = fd_precision
        desc.cpen = cpen
        desc.max_rhs = max_rhs
        desc.matvec_precision = matvec_precision
        desc.matvec_form = matvec_form
        desc.geometry_amplitude = geometry_amplitude
        desc.viscosity_contrast = viscosity_contrast
        h = ctypes.c_void_p()
        _check(lib.fdst_setup(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.max_rhs = max_rhs
        s = Sizes()
        _check(lib.fdst_get_sizes(h, ctypes.byref(s)))
        self.dim = s.dim
        self.n_total = int(s.n_total)
        self.block_offsets = [int(s.block_offset[b]) for b in range(s.nblocks)] + [self.n_total]
        self.block_shapes = [tuple(int(v) for v in s.block_shape[b]) for b in range(s.nblocks)]
        self.block_sizes = [self.block_offsets[b + 1] - self.block_offsets[b] for b in range(s.nblocks)]
        self.device_bytes = int(s.device_bytes)
        self.flops_apply = float(s.flops_apply)
        self.flops_matvec = float(s.flops_matvec)

    def close(self):
        if getattr(self, "_h", None):
            _lib.fdst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _nrhs(self, t):
        n = t.numel() // self.n_total
        if n * self.n_total != t.numel():
            raise ValueError("vector length is not a multiple of n_total")
        return n

    def apply_prec(self, r, s, stream=None):
        _check(_lib.fdst_apply_prec(self._h, _dptr(r), _dptr(s), self._nrhs(r), _stream_ptr(stream)))

    def matvec(self, x, y, stream=None):
        _check(_lib.fdst_matvec(self._h, _dptr(x), _dptr(y), self._nrhs(x), _stream_ptr(stream)))

    def apply_block_prec(self, r, s, prec=None, stream=None):
        """s = P^{-1} r for P_T (PREC_PT, default) or P_C (PREC_PC)."""
        _check(_lib.fdst_apply_block_prec(self._h, PREC_PT if prec is None else prec, _dptr(r), _dptr(s),
                                          self._nrhs(r), _stream_ptr(stream)))

    def solve_gmres(self, b, x, prec=None, form=None, tol=1e-8, maxit=1000, restart=60, stream=None, check=False):
        """GMRES with the block triangular (PREC_PT) or constraint (PREC_PC) preconditioner
        built from this handle's FD blocks (fdst_solve_gmres); form GMRES_LEFT,
        GMRES_FLEXIBLE or GMRES_AUTO (default)."""
        n = self._nrhs(b)
        info = (SolveInfo * n)()
        code = _lib.fdst_solve_gmres(self._h, PREC_PT if prec is None else prec, GMRES_AUTO if form is None else form,
                                     _dptr(b), _dptr(x), n, tol, maxit, restart, info, _stream_ptr(stream))
        if check:
            _check(code)
        return [dict(iterations=i.iterations, status=STATUS.get(i.status, i.status), eta_rel=i.eta_rel,
                     true_rel_res=i.true_rel_res, iterations_estimate=i.iterations_estimate) for i in info]

    def solve(self, b, x, tol=1e-8, maxit=1000, stream=None, check=False):
        n = self._nrhs(b)
        info = (SolveInfo * n)()
        code = _lib.fdst_solve(self._h, _dptr(b), _dptr(x), n, tol, maxit, info, _stream_ptr(stream))
        if check:
            _check(code)
        elif code not in (0, 5, 6, 7, 9):
            _check(code)
        return [dict(iterations=i.iterations, status=STATUS.get(i.status, i.status), eta_rel=i.eta_rel,
                     true_rel_res=i.true_rel_res, iterations_estimate=i.iterations_estimate) for i in info]

    def solve_host(self, b, x, tol=1e-8, maxit=1000, stream=None, zero_guess=False):
        """b, x: host numpy float64 arrays. x is the initial guess, overwritten by the
        solution; with zero_guess=True the solve starts from x0 = 0 and x is output only."""
        n = b.size // self.n_total
        info = (SolveInfo * n)()
        entry = _lib.fdst_solve_host_zero if zero_guess else _lib.fdst_solve_host
        code = entry(self._h, ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data), n,
                     tol, maxit, info, _stream_ptr(stream))
        if code not in (0, 5, 6, 7, 9):
            _check(code)
        return [dict(iterations=i.iterations, status=STATUS.get(i.status, i.status), eta_rel=i.eta_rel,
                     true_rel_res=i.true_rel_res, iterations_estimate=i.iterations_estimate) for i in info]

    def apply_prec_host(self, r, s, stream=None):
        n = r.size // self.n_total
        _check(_lib.fdst_apply_prec_host(self._h, ctypes.c_void_p(r.ctypes.data), ctypes.c_void_p(s.ctypes.data),
                                         n, _stream_ptr(stream)))

    def set_timing(self, on=True):
        _check(_lib.fdst_set_timing(self._h, int(on)))

    def get_timing(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        m, p = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.fdst_get_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(m),
                                    ctypes.byref(p)))
        k, kn = ctypes.c_double(), ctypes.c_int64()
        _check(_lib.fdst_get_kernel_timing(self._h, ctypes.byref(k), ctypes.byref(kn)))
        return dict(ms_matvec=a.value, ms_prec=b.value, ms_vector=c.value, n_matvec=m.value, n_prec=p.value,
                    ms_matvec_kernels=k.value, n_matvec_kernel_launches=kn.value)


class Batch:
    """Grouped solves of several Stokes problems (fdst_batch_*): every phase of a
    MINRES iteration is one launch over all problems, replayed from a CUDA graph."""

    def __init__(self, problems, autotune=True):
        lib = load_library()
        self.problems = list(problems)
        hs = (ctypes.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        b = ctypes.c_void_p()
        _check(lib.fdst_batch_create(hs, len(self.problems), int(autotune), ctypes.byref(b)))
        self._b = b

    def info(self):
        r, t, a, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(_lib.fdst_batch_info(self._b, ctypes.byref(r), ctypes.byref(t), ctypes.byref(a), ctypes.byref(m)))
        n = ctypes.c_int()
        _check(_lib.fdst_batch_tuning(self._b, 0, ctypes.byref(n), None, None))
        modes, rings = (ctypes.c_int * max(1, n.value))(), (ctypes.c_int * max(1, n.value))()
        _check(_lib.fdst_batch_tuning(self._b, n.value, ctypes.byref(n), modes, rings))
        return dict(tc_ring=r.value, band_threads=t.value, ms_apply=a.value, ms_matvec=m.value,
                    step_modes=[BATCH_MODES[modes[k]] for k in range(n.value)], step_rings=list(rings[:n.value]))

    def set_tuning(self, modes, rings):
        """Feeding mode ("streamed", "resident_b", "resident_b_tmem_a") and ring depth
        (0 = as deep as fits) of every contraction step."""
        codes = {v: k for k, v in BATCH_MODES.items()}
        if len(modes) != len(rings) or any(m not in codes or codes[m] == 0 for m in modes):
            raise ValueError("modes: one of streamed / resident_b / resident_b_tmem_a per step, rings alike")
        n = len(modes)
        cm, cr = (ctypes.c_int * max(1, n))(*[codes[m] for m in modes]), (ctypes.c_int * max(1, n))(*rings)
        _check(_lib.fdst_batch_set_tuning(self._b, n, cm, cr))

    def solve(self, bs, xs, tol=1e-8, maxit=1000, stream=None):
        n = len(self.problems)
        bp = (ctypes.c_void_p * n)(*[_dptr(v).value for v in bs])
        xp = (ctypes.c_void_p * n)(*[_dptr(v).value for v in xs])
        info = (SolveInfo * n)()
        code = _lib.fdst_batch_solve(self._b, bp, xp, tol, maxit, info, _stream_ptr(stream))
        if code not in (0, 5, 6, 7, 9):
            _check(code)
        return [dict(iterations=i.iterations, status=STATUS.get(i.status, i.status), eta_rel=i.eta_rel,
                     true_rel_res=i.true_rel_res, iterations_estimate=i.iterations_estimate) for i in info]

    def close(self):
        if getattr(self, "_b", None):
            _lib.fdst_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc_for(knots, p, disc=TH, viscosity=1.0, cpen=0.0):
    keep = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    d = Desc()
    d.dim = len(keep)
    d.discretization = disc
    d.degree = p
    for e, k in enumerate(keep):
        d.h_knots[e] = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.nknots[e] = len(k)
    d.viscosity = viscosity
    d.cpen = cpen
    d.max_rhs = 1
    return d, keep


class Server:
    """Continuous-batching request server (fdst_server_*). Times are the caller's clock."""

    def __init__(self, max_active=16, hbm_budget_bytes=0, fd_precision=FD_TF32X3, matvec_precision=MV_DF64,
                 tol=1e-8, maxit=1000, iters_per_step=4):
        lib = load_library()
        o = ServerOpts(hbm_budget_bytes, max_active, fd_precision, matvec_precision, tol, maxit, iters_per_step)
        s = ctypes.c_void_p()
        _check(lib.fdst_server_create(ctypes.byref(o), ctypes.byref(s)))
        self._s = s
        self.sizes = {}

    def submit(self, knots, p, b, t_arrival, disc=TH):
        d, keep = _desc_for(knots, p, disc)
        b = np.ascontiguousarray(b, dtype=np.float64)
        rid = ctypes.c_int64()
        _check(_lib.fdst_server_submit(self._s, ctypes.byref(d), ctypes.c_void_p(b.ctypes.data), t_arrival,
                                       ctypes.byref(rid)))
        self.sizes[rid.value] = b.size
        return rid.value

    def step(self, now):
        a, q, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(_lib.fdst_server_step(self._s, now, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)))
        return a.value, q.value, f.value

    def result(self, rid):
        fin = ctypes.c_int()
        x = np.empty(self.sizes[rid])
        info = SolveInfo()
        ta, tm, td = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(_lib.fdst_server_result(self._s, rid, ctypes.byref(fin), ctypes.c_void_p(x.ctypes.data),
                                       ctypes.byref(info), ctypes.byref(ta), ctypes.byref(tm), ctypes.byref(td)))
        if not fin.value:
            return None
        return dict(x=x, iterations=info.iterations, status=STATUS.get(info.status, info.status),
                    true_rel_res=info.true_rel_res, t_arrival=ta.value, t_admit=tm.value, t_done=td.value)

    def cancel(self, rid):
        """Withdraw a request: a queued one finishes at once, an active one at the next step (CANCELLED)."""
        _check(_lib.fdst_server_cancel(self._s, rid))

    def stats(self):
        c, r, e, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        m = ctypes.c_int()
        _check(_lib.fdst_server_stats(self._s, ctypes.byref(c), ctypes.byref(r), ctypes.byref(e), ctypes.byref(b),
                                      ctypes.byref(m)))
        return dict(handles_created=c.value, handles_reused=r.value, handles_evicted=e.value, bytes_held=b.value,
                    max_active_seen=m.value)

    def close(self):
        if getattr(self, "_s", None):
            _lib.fdst_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
