"""Thin ctypes binding of the C ABI in ``include/abc.h`` (argument marshalling only).

Every step of the path runs in the native library; this module checks tensor
dtypes / shapes / devices, passes raw pointers and raises ``AbcError`` on a
non-zero status.  The library must have been built (``build.build()``); there is
no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

OK = 0
FP64, C64_FP32, C64_SPLIT_BF16, C64_3XTF32, C64_SPLIT_FP16 = 0, 1, 2, 3, 4
MAT_K, MAT_M, MAT_A, MAT_B, MAT_Q = 0, 1, 2, 3, 4
MAT_B1, MAT_B0, MAT_A1, MAT_A0 = 5, 6, 7, 8
KERNEL_CONTRACTION, KERNEL_STENCIL, KERNEL_PACK = 0, 1, 2
TUNE_L2_KEEP_TILES, TUNE_TILE_COUNT, TUNE_PDL, TUNE_CHAIN, TUNE_STENCIL, TUNE_FUSED = 0, 1, 2, 3, 4, 5
TUNE_GEMM_TILE, TUNE_GEMM_SPLIT, TUNE_STENCIL_BPS, TUNE_STENCIL_KZ, TUNE_BACK_MULTI = 6, 7, 8, 9, 10
TUNE_FORWARD_RW, TUNE_GAMMA_COPY, TUNE_STENCIL_STAGED, TUNE_LANES = 11, 12, 13, 14
PRECISIONS = {"fp64": FP64, "c64": C64_FP32, "bf16x3": C64_SPLIT_BF16, "tf32x3": C64_3XTF32,
              "fp16x3": C64_SPLIT_FP16}
FIT1_LIMIT, FIT1_TWO_POINT, FIT1_HERMITE = 0, 1, 2
FITS1 = {"limit": FIT1_LIMIT, "two_point": FIT1_TWO_POINT, "hermite": FIT1_HERMITE}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libabc.so")


class AbcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class abc_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("radius", ctypes.c_int), ("h", ctypes.c_double)]


class abc_params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("s0", ctypes.c_double), ("s1", ctypes.c_double),
                ("precision", ctypes.c_int), ("max_orbitals", ctypes.c_int), ("s2", ctypes.c_double * 4),
                ("fit1", ctypes.c_int), ("s1b", ctypes.c_double)]


class abc_meanfield(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("alpha", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def load():
    """Load the native library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"native library not built: {LIB_PATH} (run paper_1908_02456_gb300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    G, Pm, MF = ctypes.POINTER(abc_grid), ctypes.POINTER(abc_params), ctypes.POINTER(abc_meanfield)
    sig = {
        "abc_setup": [G, Pm, ctypes.POINTER(_P)],
        "abc_boundary_size": [_P, ctypes.POINTER(ctypes.c_longlong)],
        "abc_step": [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, _P],
        "abc_run": [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, MF, ctypes.c_int, _P, _P],
        "abc_run_host": [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, MF, ctypes.c_int, _P],
        "abc_diagnostics": [_P, _P, _P, _P, ctypes.c_int, MF, _P, _P],
        "abc_adjoint_run": [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_int, _P, _P, _P],
        "abc_get_matrices": [_P, ctypes.c_int, _P, ctypes.c_size_t],
        "abc_wait_selftest": [_P, ctypes.c_longlong, _P],
        "abc_host_matrices": [G, Pm, ctypes.c_int, _P, ctypes.c_size_t],
        "abc_profile_enable": [_P, ctypes.c_int],
        "abc_profile_read": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)],
        "abc_profile_durations": [_P, ctypes.c_int, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)],
        "abc_kernel_bytes": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
        "abc_kernel_flops": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)],
        "abc_state_size": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "abc_get_state": [_P, _P, _P, ctypes.c_int, _P, ctypes.c_size_t, _P],
        "abc_set_state": [_P, _P, _P, ctypes.c_int, _P, ctypes.c_size_t, _P],
        "abc_progress": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)],
        "abc_launch_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
        "abc_step_noalloc": [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, _P],
        "abc_set_tuning": [_P, ctypes.c_int, ctypes.c_longlong],
        "abc_aux_init": [_P, _P, _P, ctypes.c_int, _P],
        "abc_get_tuning": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.abc_destroy.argtypes = [_P]
    lib.abc_destroy.restype = None
    lib.abc_status_string.argtypes = [ctypes.c_int]
    lib.abc_status_string.restype = ctypes.c_char_p
    lib.abc_last_error.argtypes = []
    lib.abc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int):
    if st != OK:
        lib = load()
        raise AbcError(st, f"{lib.abc_status_string(st).decode()}: {lib.abc_last_error().decode()}")


def _grid(shape: Sequence[int], h: float, radius: int = 1) -> abc_grid:
    nx, ny, nz = (int(v) for v in shape)
    return abc_grid(nx, ny, nz, int(radius), float(h))


def _params(order: int, s, precision, max_orbitals: int, fit1="limit", s1b: float = 0.0) -> abc_params:
    """s: the interpolation point (orders 0, 1) or the four points (order 2); fit1 (order 1):
    "limit" (Thm 3.2), "two_point" (with the second point s1b) or "hermite" (eq:39)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    fit = FITS1[fit1] if isinstance(fit1, str) else int(fit1)
    if int(order) == 2:
        pts = [float(v) for v in s]
        if len(pts) != 4:
            raise ValueError("order 2 needs four interpolation points")
        return abc_params(2, pts[0], pts[0], prec, int(max_orbitals), (ctypes.c_double * 4)(*pts), fit,
                          float(s1b))
    return abc_params(int(order), float(s), float(s), prec, int(max_orbitals), (ctypes.c_double * 4)(0, 0, 0, 0),
                      fit, float(s1b))


def _mf(meanfield) -> Optional[ctypes.POINTER(abc_meanfield)]:
    if meanfield is None:
        return None
    a, b, alpha = meanfield
    return ctypes.pointer(abc_meanfield(float(a), float(b), float(alpha)))


# ----------------------------------------------------------------------
# the C functions under their own names
# ----------------------------------------------------------------------
def abc_setup(grid: abc_grid, params: abc_params) -> ctypes.c_void_p:
    ctx = _P()
    _check(load().abc_setup(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(ctx)))
    return ctx


def abc_boundary_size(ctx) -> int:
    n = ctypes.c_longlong()
    _check(load().abc_boundary_size(ctx, ctypes.byref(n)))
    return n.value


def abc_step(ctx, psi_ptr: int, aux_ptr: int, V_ptr: int, n_orb: int, dt: float, stream: int = 0):
    _check(load().abc_step(ctx, psi_ptr, aux_ptr or None, V_ptr, n_orb, dt, stream or None))


def abc_run(ctx, psi_ptr, aux_ptr, V_ptr, n_orb, dt, nsteps, meanfield=None, diag_every=0, diag_out=None,
            stream: int = 0):
    d = None if diag_out is None else diag_out.ctypes.data_as(_P)
    _check(load().abc_run(ctx, psi_ptr, aux_ptr or None, V_ptr, n_orb, dt, nsteps, _mf(meanfield), diag_every, d,
                          stream or None))


def abc_run_host(ctx, psi: np.ndarray, aux: Optional[np.ndarray], V: np.ndarray, n_orb, dt, nsteps,
                 meanfield=None, diag_every=0, diag_out=None):
    d = None if diag_out is None else diag_out.ctypes.data_as(_P)
    _check(load().abc_run_host(ctx, psi.ctypes.data_as(_P), None if aux is None else aux.ctypes.data_as(_P),
                               V.ctypes.data_as(_P), n_orb, dt, nsteps, _mf(meanfield), diag_every, d))


def abc_diagnostics(ctx, psi_ptr, aux_ptr, V_ptr, n_orb, meanfield=None, stream: int = 0) -> np.ndarray:
    out = np.zeros((n_orb, 3))
    _check(load().abc_diagnostics(ctx, psi_ptr, aux_ptr or None, V_ptr, n_orb, _mf(meanfield),
                                  out.ctypes.data_as(_P), stream or None))
    return out


def abc_adjoint_run(ctx, psi0_ptr, V_ptr, n_orb, dt, nsteps, ckpt_every, dJdV_ptr, stream: int = 0) -> float:
    J = ctypes.c_double()
    _check(load().abc_adjoint_run(ctx, psi0_ptr, V_ptr, n_orb, dt, nsteps, ckpt_every, ctypes.byref(J), dJdV_ptr,
                                  stream or None))
    return J.value


def abc_wait_selftest(ctx, polls: int, stream=None) -> int:
    """Status of the bounded-wait self-test (ABC_ERR_TIMEOUT = 5 when the path works)."""
    return int(load().abc_wait_selftest(ctx, int(polls), stream))


def abc_get_matrices(ctx, which: int, n_gamma: int) -> np.ndarray:
    out = np.zeros((n_gamma, n_gamma), np.complex128)
    _check(load().abc_get_matrices(ctx, which, out.ctypes.data_as(_P), out.nbytes))
    return out


def abc_host_matrices(shape, h, order, s, which, fit1="limit", s1b: float = 0.0, radius: int = 1) -> np.ndarray:
    """FP64 setup on the host only (no CUDA): dense ABC_MAT_* in natural Gamma order."""
    nx, ny, nz = shape
    R = int(radius)
    n = nx * ny * nz - max(nx - 2 * R, 0) * max(ny - 2 * R, 0) * max(nz - 2 * R, 0)
    out = np.zeros((n, n), np.complex128)
    g, p = _grid(shape, h, radius), _params(order, s, FP64, 1, fit1, s1b)
    _check(load().abc_host_matrices(ctypes.byref(g), ctypes.byref(p), which, out.ctypes.data_as(_P), out.nbytes))
    return out


def abc_profile_enable(ctx, enable: bool):
    _check(load().abc_profile_enable(ctx, int(bool(enable))))


def abc_profile_read(ctx, kernel: int):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load().abc_profile_read(ctx, kernel, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def abc_profile_durations(ctx, kernel: int, max_out: int = 1 << 16) -> np.ndarray:
    out = np.zeros(max_out, np.float32)
    n = ctypes.c_longlong()
    _check(load().abc_profile_durations(ctx, kernel, out.ctypes.data_as(_P), max_out, ctypes.byref(n)))
    return out[:min(n.value, max_out)].copy()


def abc_kernel_bytes(ctx, kernel: int, n_orb: int) -> float:
    b = ctypes.c_double()
    _check(load().abc_kernel_bytes(ctx, kernel, n_orb, ctypes.byref(b)))
    return b.value


def abc_kernel_flops(ctx, kernel: int, n_orb: int):
    """(useful, issued) flops of one contraction launch."""
    u, i = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().abc_kernel_flops(ctx, kernel, n_orb, ctypes.byref(u), ctypes.byref(i)))
    return u.value, i.value


def abc_state_size(ctx, n_orb: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().abc_state_size(ctx, n_orb, ctypes.byref(n)))
    return n.value


def abc_get_state(ctx, psi_ptr, aux_ptr, n_orb, stream: int = 0) -> np.ndarray:
    """The state blob (uint8 array) of psi / aux on the device."""
    buf = np.empty(abc_state_size(ctx, n_orb), dtype=np.uint8)
    _check(load().abc_get_state(ctx, psi_ptr, aux_ptr or None, n_orb, buf.ctypes.data, buf.nbytes, stream or None))
    return buf


def abc_set_state(ctx, psi_ptr, aux_ptr, n_orb, blob: np.ndarray, stream: int = 0):
    blob = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(load().abc_set_state(ctx, psi_ptr, aux_ptr or None, n_orb, blob.ctypes.data, blob.nbytes, stream or None))


def abc_progress(ctx):
    n, t = ctypes.c_longlong(0), ctypes.c_double(0)
    _check(load().abc_progress(ctx, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def abc_set_tuning(ctx, key: int, value: int):
    _check(load().abc_set_tuning(ctx, key, int(value)))


def abc_get_tuning(ctx, key: int) -> int:
    v = ctypes.c_longlong()
    _check(load().abc_get_tuning(ctx, key, ctypes.byref(v)))
    return v.value


def abc_launch_count(ctx) -> int:
    n = ctypes.c_longlong()
    _check(load().abc_launch_count(ctx, ctypes.byref(n)))
    return n.value


def abc_destroy(ctx):
    if ctx:
        load().abc_destroy(ctx)


# ----------------------------------------------------------------------
# convenience wrapper over torch tensors
# ----------------------------------------------------------------------
class Context:
    """Owns one abc_ctx.  psi: [b, nz, ny, nx] complex CUDA tensor; aux: [n_gamma, b]."""

    def __init__(self, shape, h, order, s, precision="c64", max_orbitals=1, fit1="limit", s1b=0.0, radius=1):
        self.shape = tuple(int(v) for v in shape)
        self.h, self.order = float(h), int(order)
        self.s = tuple(float(v) for v in s) if self.order == 2 else float(s)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.max_orbitals = int(max_orbitals)
        self.fit1 = FITS1[fit1] if isinstance(fit1, str) else int(fit1)
        self.s1b = float(s1b)
        self.radius = int(radius)
        self.ctx = abc_setup(_grid(self.shape, h, self.radius),
                             _params(order, s, self.precision, max_orbitals, self.fit1, self.s1b))
        self.n_gamma = abc_boundary_size(self.ctx)

    # dtypes of the path
    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == FP64 else torch.complex64

    @property
    def real_dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def _check_tensors(self, psi, aux, V):
        nx, ny, nz = self.shape
        if not psi.is_cuda or psi.dtype != self.complex_dtype or not psi.is_contiguous():
            raise ValueError(f"psi must be a contiguous CUDA {self.complex_dtype} tensor")
        if psi.dim() != 4 or tuple(psi.shape[1:]) != (nz, ny, nx):
            raise ValueError(f"psi must have shape [b, {nz}, {ny}, {nx}]")
        b = psi.shape[0]
        if self.order >= 1:
            shp = self.aux_shape(b)
            if aux is None or not aux.is_cuda or aux.dtype != self.complex_dtype or not aux.is_contiguous() \
                    or tuple(aux.shape) != shp:
                raise ValueError(f"aux must be a contiguous CUDA {self.complex_dtype} tensor {list(shp)}")
        if not V.is_cuda or V.dtype != self.real_dtype or not V.is_contiguous() or tuple(V.shape) != (nz, ny, nx):
            raise ValueError(f"V must be a contiguous CUDA {self.real_dtype} tensor [{nz}, {ny}, {nx}]")
        return b

    @staticmethod
    def _stream(stream):
        import torch
        return (stream or torch.cuda.current_stream()).cuda_stream

    def aux_shape(self, b):
        """[n_gamma, b] (order 1: f) or [2, n_gamma, b] (order 2: f then g = df/dt)."""
        return (2, self.n_gamma, b) if self.order == 2 else (self.n_gamma, b)

    def new_aux(self, b):
        """Zero auxiliary state (order 1 starts there; order 2 needs init_aux)."""
        import torch
        return torch.zeros(self.aux_shape(b), dtype=self.complex_dtype, device="cuda")

    def init_aux(self, psi, stream=None):
        """Consistent auxiliary state at t = 0 for psi (abc_aux_init); None for order 0."""
        if self.order == 0:
            return None
        aux = self.new_aux(psi.shape[0])
        _check(load().abc_aux_init(self.ctx, psi.data_ptr(), aux.data_ptr(), psi.shape[0], self._stream(stream)))
        return aux

    def step(self, psi, aux, V, dt, stream=None):
        b = self._check_tensors(psi, aux, V)
        abc_step(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else 0, V.data_ptr(), b, dt,
                 self._stream(stream))

    def run(self, psi, aux, V, dt, nsteps, meanfield=None, diag_every=0, stream=None):
        b = self._check_tensors(psi, aux, V)
        diag = np.zeros((nsteps // diag_every, b, 3)) if diag_every else None
        abc_run(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else 0, V.data_ptr(), b, dt, nsteps,
                meanfield, diag_every, diag, self._stream(stream))
        return diag

    def run_host(self, psi, aux, V, dt, nsteps, meanfield=None, diag_every=0):
        """Host buffers (numpy arrays or CPU torch tensors, e.g. pinned); copies in,
        runs, copies back into psi / aux."""
        def host(x):
            if x is None:
                return None
            if isinstance(x, np.ndarray):
                return x
            if x.is_cuda or not x.is_contiguous():
                raise ValueError("run_host needs contiguous host tensors")
            return x.numpy()
        psi_h, aux_h, V_h = host(psi), host(aux), host(V)
        b = psi_h.shape[0]
        diag = np.zeros((nsteps // diag_every, b, 3)) if diag_every else None
        abc_run_host(self.ctx, psi_h, aux_h, V_h, b, dt, nsteps, meanfield, diag_every, diag)
        return diag

    def diagnostics(self, psi, aux, V, meanfield=None, stream=None):
        b = self._check_tensors(psi, aux, V)
        return abc_diagnostics(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else 0, V.data_ptr(), b,
                               meanfield, self._stream(stream))

    def adjoint(self, psi0, V, dt, nsteps, ckpt_every=50, stream=None):
        import torch
        b = self._check_tensors(psi0, self.new_aux(psi0.shape[0]) if self.order == 1 else None, V)
        g = torch.empty_like(V)
        J = abc_adjoint_run(self.ctx, psi0.data_ptr(), V.data_ptr(), b, dt, nsteps, ckpt_every, g.data_ptr(),
                            self._stream(stream))
        return J, g

    def matrix(self, which):
        return abc_get_matrices(self.ctx, which, self.n_gamma)

    def profile(self, enable=True):
        abc_profile_enable(self.ctx, enable)

    def profile_read(self, kernel=KERNEL_CONTRACTION):
        return abc_profile_read(self.ctx, kernel)

    def profile_durations(self, kernel=KERNEL_CONTRACTION):
        return abc_profile_durations(self.ctx, kernel)

    def kernel_bytes(self, kernel, n_orb):
        return abc_kernel_bytes(self.ctx, kernel, n_orb)

    def get_state(self, psi, aux, stream=None) -> np.ndarray:
        """Checkpoint blob of (psi, aux) and the context's progress."""
        b = psi.shape[0]
        return abc_get_state(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else 0, b,
                             self._stream(stream))

    def set_state(self, psi, aux, blob, stream=None):
        """Restore (psi, aux) in place from a checkpoint blob (validated by the library)."""
        b = psi.shape[0]
        abc_set_state(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else 0, b, blob,
                      self._stream(stream))

    def progress(self):
        return abc_progress(self.ctx)

    def kernel_flops(self, kernel, n_orb):
        return abc_kernel_flops(self.ctx, kernel, n_orb)

    def set_tuning(self, key, value):
        abc_set_tuning(self.ctx, key, value)

    def get_tuning(self, key):
        return abc_get_tuning(self.ctx, key)

    def launches(self):
        return abc_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            abc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------
# the one-dimensional stepper of Sec. 4.1 (include/abc1d.h)
# ----------------------------------------------------------------------
class abc1d_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("h", ctypes.c_double), ("order", ctypes.c_int),
                ("s", ctypes.c_double * 4), ("fit1", ctypes.c_int), ("precision", ctypes.c_int)]


def _params1d(n, h, order, s, fit1="limit", precision="fp64") -> abc1d_params:
    pts = [float(v) for v in (s if isinstance(s, (tuple, list)) else (s,))] + [0.0] * 4
    fit = FITS1[fit1] if isinstance(fit1, str) else int(fit1)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return abc1d_params(int(n), float(h), int(order), (ctypes.c_double * 4)(*pts[:4]), fit, prec)


def _sig1d(lib):
    P1 = ctypes.POINTER(abc1d_params)
    for name, args in {"abc1d_setup": [P1, ctypes.POINTER(_P)], "abc1d_aux_init": [_P, _P, _P, _P],
                       "abc1d_run": [_P, _P, _P, ctypes.c_double, ctypes.c_longlong, ctypes.c_int, _P, _P],
                       "abc1d_host_block": [P1, ctypes.c_int, _P], "abc1d_destroy": [_P]}.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None if name == "abc1d_destroy" else ctypes.c_int


def abc1d_host_block(n, h, order, s, which, fit1="limit") -> np.ndarray:
    """The left end's 2 x 2 block of matrix `which` (GPU-free set-up)."""
    lib = load()
    _sig1d(lib)
    out = np.zeros(8)
    p = _params1d(n, h, order, s, fit1)
    _check(lib.abc1d_host_block(ctypes.byref(p), which, out.ctypes.data))
    return out.view(np.complex128).reshape(2, 2)


class Context1D:
    """One abc1d_ctx: psi is a CUDA tensor of n complex values, aux of 4 (order 1) or 8
    (order 2: f then g)."""

    def __init__(self, n, h, order, s, fit1="limit", precision="fp64"):
        lib = load()
        _sig1d(lib)
        self.n, self.h, self.order = int(n), float(h), int(order)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p = _params1d(n, h, order, s, fit1, precision)
        c = _P()
        _check(lib.abc1d_setup(ctypes.byref(p), ctypes.byref(c)))
        self.ctx = c

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == FP64 else torch.complex64

    def new_aux(self, psi):
        """The consistent auxiliary state at t = 0 (None for order 0)."""
        import torch
        if self.order == 0:
            return None
        aux = torch.zeros(4 if self.order == 1 else 8, dtype=self.complex_dtype, device="cuda")
        _check(load().abc1d_aux_init(self.ctx, psi.data_ptr(), aux.data_ptr(), None))
        return aux

    def run(self, psi, aux, dt, nsteps, diag_every=0):
        if psi.dtype != self.complex_dtype or not psi.is_cuda or psi.numel() != self.n or not psi.is_contiguous():
            raise ValueError(f"psi must be a contiguous CUDA {self.complex_dtype} tensor of {self.n} values")
        norms = np.zeros(nsteps // diag_every) if diag_every else None
        _check(load().abc1d_run(self.ctx, psi.data_ptr(), aux.data_ptr() if aux is not None else None, dt, nsteps,
                                diag_every, norms.ctypes.data if norms is not None else None, None))
        return norms

    def close(self):
        if getattr(self, "ctx", None):
            load().abc1d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
