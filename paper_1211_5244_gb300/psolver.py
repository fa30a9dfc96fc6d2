"""Thin ctypes binding of libpsolver (include/psolver.h), same names as the C ABI.

Only marshals arguments: every step of a solve runs in the library's CUDA
kernels. PyTorch provides device memory and streams. There is no fallback:
if the library is not built, ``load_library`` raises.

Arrays are torch tensors of shape (n3, n2, n1), contiguous, x fastest, on the
device the plan was built on, with the plan's dtype (float32 or float64).
Boundary conditions are a 3-letter string for the x, y, z axes: 'p' periodic,
'f' free (e.g. "pff" = wire periodic along x).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PS_BC_PERIODIC, PS_BC_FREE = 0, 1
PS_F32, PS_F64 = 0, 1
PS_MATH_CUDACORE, PS_MATH_TF32X3, PS_MATH_BF16X3 = 0, 1, 2
STATUS = {0: "PS_OK", 1: "PS_ERR_ARG", 2: "PS_ERR_UNSUPPORTED", 3: "PS_ERR_NOT_BUILT",
          4: "PS_ERR_CUDA", 5: "PS_ERR_OOM", 6: "PS_ERR_TIMEOUT"}

_lib = None


class PsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 3), ("L", ctypes.c_int * 3),
        ("c", ctypes.c_int), ("dtype", ctypes.c_int), ("math", ctypes.c_int),
        ("lines", ctypes.c_longlong * 5), ("line_len", ctypes.c_longlong * 5),
        ("fft_points", ctypes.c_double), ("paper_points", ctypes.c_double),
        ("paper_full_points", ctypes.c_double), ("alg_bytes", ctypes.c_double),
        ("workspace_bytes", ctypes.c_size_t), ("launches", ctypes.c_int),
        ("tensor_passes", ctypes.c_int), ("blocks", ctypes.c_int * 5), ("fused", ctypes.c_int),
        ("order", ctypes.c_int * 3), ("schedule", ctypes.c_int * 6), ("chunks", ctypes.c_int),
        ("axis_schedule", (ctypes.c_int * 2) * 3),
    ]


def library_path():
    return _build.LIB


def load_library():
    """Loads the in-tree libpsolver.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libpsolver.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ps_plan_create": [i, i, i, d, i, i, i, i, ctypes.POINTER(vp)],
        "ps_plan_set_lengths": [vp, i, i, i],
        "ps_plan_set_math": [vp, i],
        "ps_plan_set_schedule": [vp, i, i, i, i, i, i],
        "ps_plan_set_axis_schedule": [vp, i, i, i],
        "ps_plan_set_order": [vp, i, i, i],
        "ps_plan_autotune": [vp, i, vp],
        "ps_plan_query": [vp, ctypes.POINTER(PlanInfo)],
        "ps_kernel_build": [vp, vp],
        "ps_kernel_get": [vp, vp, vp],
        "ps_kernel_set_real": [vp, vp, vp],
        "ps_solve": [vp, vp, vp, vp, vp],
        "ps_solve_adjoint": [vp, vp, vp, vp],
        "ps_solve_vjp": [vp, vp, vp, vp, vp, vp],
        "ps_solve_batched": [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp],
        "ps_solve_host": [vp, vp, vp, vp, vp],
        "ps_solve_host_stream": [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp],
        "ps_plan_set_profiling": [vp, i],
        "ps_plan_pass_times": [vp, ctypes.POINTER(d), ctypes.POINTER(i)],
        "ps_plan_device_status": [vp, vp],
        "ps_plan_destroy": [vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = i
    lib.ps_hartree_energy_noalloc.argtypes = [i, ctypes.c_longlong, d, vp, vp, vp, vp]
    lib.ps_hartree_energy_noalloc.restype = i
    lib.ps_strerror.argtypes = [i]
    lib.ps_strerror.restype = ctypes.c_char_p
    lib.ps_last_error.argtypes = []
    lib.ps_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        msg = _lib.ps_last_error().decode(errors="replace")
        raise PsError(code, msg or _lib.ps_strerror(code).decode())


def _bc_codes(bc):
    bc = str(bc).lower()
    if len(bc) != 3 or any(b not in "pf" for b in bc):
        raise ValueError(f"bc must be 3 letters of 'p'/'f', got {bc!r}")
    return [PS_BC_PERIODIC if b == "p" else PS_BC_FREE for b in bc]


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """One solve geometry: ps_plan_create (+ optional lengths) and ps_kernel_build."""

    def __init__(self, n, bc, h, dtype="f32", L=None, build=True, stream=None, autotune=False,
                 math="cudacore", schedule=None, order=None, axis_schedule=None):
        lib = load_library()
        self.n = tuple(int(v) for v in n)
        self.bc = str(bc).lower()
        self.h = float(h)
        self.dtype = {"f32": PS_F32, "float32": PS_F32, "f64": PS_F64, "float64": PS_F64}[str(dtype)]
        handle = ctypes.c_void_p()
        codes = _bc_codes(bc)
        _check(lib.ps_plan_create(self.n[0], self.n[1], self.n[2], self.h, codes[0], codes[1], codes[2],
                                  self.dtype, ctypes.byref(handle)))
        self._h = handle
        if L is not None:
            _check(lib.ps_plan_set_lengths(self._h, int(L[0]), int(L[1]), int(L[2])))
        self.math = {"cudacore": PS_MATH_CUDACORE, "tf32x3": PS_MATH_TF32X3,
                     "bf16x3": PS_MATH_BF16X3}[str(math).lower()]
        _check(lib.ps_plan_set_math(self._h, self.math))
        if order is not None:
            _check(lib.ps_plan_set_order(self._h, int(order[0]), int(order[1]), int(order[2])))
        if schedule is not None:
            self.set_schedule(**schedule)
        for axis, sched in (axis_schedule or {}).items():
            self.set_axis_schedule(axis, **sched)
        if autotune:
            _check(lib.ps_plan_autotune(self._h, 5, _stream_handle(stream)))
        if build:
            self.build(stream)

    def set_schedule(self, tile=0, radix=0, ztk=0, ykind=0, xy=0, chunks=0):
        """ps_plan_set_schedule: the kernel schedule by hand (before the build)."""
        _check(_lib.ps_plan_set_schedule(self._h, int(tile), int(radix), int(ztk), int(ykind), int(xy),
                                         int(chunks)))
        return self

    def set_axis_schedule(self, axis, tile=0, radix=-1):
        """ps_plan_set_axis_schedule: generic tile and radix split along one axis."""
        _check(_lib.ps_plan_set_axis_schedule(self._h, int(axis), int(tile), int(radix)))
        return self

    # ------------------------------------------------------------ lifecycle
    def build(self, stream=None):
        _check(_lib.ps_kernel_build(self._h, _stream_handle(stream)))
        return self

    def close(self):
        if getattr(self, "_h", None):
            _lib.ps_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self):
        out = PlanInfo()
        _check(_lib.ps_plan_query(self._h, ctypes.byref(out)))
        return out

    @property
    def torch_dtype(self):
        import torch
        return torch.float32 if self.dtype == PS_F32 else torch.float64

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def _check_tensor(self, t, name):
        if tuple(t.shape) != self.shape or t.dtype != self.torch_dtype or not t.is_cuda \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.torch_dtype} tensor of shape "
                             f"{self.shape}, got {tuple(t.shape)} {t.dtype} on {t.device}")

    def set_profiling(self, enable=True):
        """ps_plan_set_profiling: per-pass CUDA events on every later solve."""
        _check(_lib.ps_plan_set_profiling(self._h, 1 if enable else 0))

    def device_status(self, stream=None):
        """ps_plan_device_status: raises PsError (PS_ERR_TIMEOUT) if a bounded
        device wait gave up since the last call; synchronises the stream."""
        _check(_lib.ps_plan_device_status(self._h, _stream_handle(stream)))

    def pass_times(self):
        """ps_plan_pass_times: (summed ms per pass [5], number of solves)."""
        ms = (ctypes.c_double * 5)()
        cnt = ctypes.c_int(0)
        _check(_lib.ps_plan_pass_times(self._h, ms, ctypes.byref(cnt)))
        return list(ms), cnt.value

    # ------------------------------------------------------------ solves
    def solve(self, rho, V=None, energy=True, stream=None, E=None):
        """ps_solve: returns (V, E) with E a 0-d float64 CUDA tensor (or None).
        ``V`` and ``E`` may be given as preallocated outputs."""
        import torch
        self._check_tensor(rho, "rho")
        if V is None:
            V = torch.empty_like(rho)
        self._check_tensor(V, "V")
        if energy and E is None:
            E = torch.empty((), dtype=torch.float64, device=rho.device)
        if not energy:
            E = None
        elif E.dtype != torch.float64 or not E.is_cuda or E.numel() != 1:
            raise ValueError("E must be a one-element float64 CUDA tensor")
        _check(_lib.ps_solve(self._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                             ctypes.c_void_p(E.data_ptr()) if E is not None else None,
                             _stream_handle(stream)))
        return V, E

    def solve_adjoint(self, vbar, out=None, stream=None):
        """ps_solve_adjoint: rhobar = K^T vbar (= K vbar, K is symmetric)."""
        import torch
        self._check_tensor(vbar, "vbar")
        if out is None:
            out = torch.empty_like(vbar)
        _check(_lib.ps_solve_adjoint(self._h, ctypes.c_void_p(vbar.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def solve_vjp(self, vbar=None, V=None, gE=None, out=None, stream=None):
        """ps_solve_vjp: rhobar = K vbar + h^3 gE V (terms given as None are omitted)."""
        import torch
        ref = vbar if vbar is not None else V
        if ref is None:
            raise ValueError("vbar or (V, gE) must be given")
        for t, nm in ((vbar, "vbar"), (V, "V")):
            if t is not None:
                self._check_tensor(t, nm)
        if (V is None) != (gE is None):
            raise ValueError("V and gE must be given together")
        if gE is not None and (gE.dtype != torch.float64 or not gE.is_cuda or gE.numel() != 1):
            raise ValueError("gE must be a one-element float64 CUDA tensor")
        if out is None:
            out = torch.empty_like(ref)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(_lib.ps_solve_vjp(self._h, ptr(vbar), ptr(V), ptr(gE), ptr(out), _stream_handle(stream)))
        return out

    def solve_host(self, rho_host, V_host=None, stream=None):
        """ps_solve_host on CPU tensors (pinned for asynchronous copies)."""
        import torch
        if tuple(rho_host.shape) != self.shape or rho_host.dtype != self.torch_dtype \
                or rho_host.is_cuda or not rho_host.is_contiguous():
            raise ValueError("rho_host must be a contiguous CPU tensor of the plan's shape and dtype")
        if V_host is None:
            V_host = torch.empty_like(rho_host)
        E = ctypes.c_double(0.0)
        _check(_lib.ps_solve_host(self._h, ctypes.c_void_p(rho_host.data_ptr()),
                                  ctypes.c_void_p(V_host.data_ptr()), ctypes.byref(E),
                                  _stream_handle(stream)))
        return V_host, E.value

    def solve_host_stream(self, rho_hosts, V_hosts=None, energy=True, stream=None):
        """ps_solve_host_stream: many host densities with overlapped transfers.
        Returns (V_hosts, energies) with energies a list of floats (or None)."""
        import torch
        count = len(rho_hosts)
        for r in rho_hosts:
            if tuple(r.shape) != self.shape or r.dtype != self.torch_dtype or r.is_cuda or not r.is_contiguous():
                raise ValueError("rho_hosts must be contiguous CPU tensors of the plan's shape and dtype")
        if V_hosts is None:
            V_hosts = [torch.empty_like(r) for r in rho_hosts]
        arr = ctypes.c_void_p * max(count, 1)
        rp = arr(*[r.data_ptr() for r in rho_hosts])
        vp = arr(*[v.data_ptr() for v in V_hosts])
        E = (ctypes.c_double * max(count, 1))() if energy else None
        _check(_lib.ps_solve_host_stream(self._h, count, rp, vp, E, _stream_handle(stream)))
        return V_hosts, (list(E)[:count] if energy else None)

    def set_kernel_real(self, kernel, stream=None):
        """ps_kernel_set_real: use a caller's even real-space kernel, given as a
        float64 array of shape (L3//2 + 1, L2//2 + 1, L1//2 + 1) of the values at
        the offsets (d1, d2, d3), for every later solve."""
        import numpy as np
        L = self.info().L
        want = (L[2] // 2 + 1, L[1] // 2 + 1, L[0] // 2 + 1)
        k = np.ascontiguousarray(kernel, dtype=np.float64)
        if k.shape != want:
            raise ValueError(f"kernel octant must have shape {want}, got {k.shape}")
        _check(_lib.ps_kernel_set_real(self._h, k.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return self

    def kernel_octant(self, stream=None):
        """ps_kernel_get: the stored K^F / (L1 L2 L3) octant, shape (L3/2+1, L2/2+1, c)."""
        import torch
        inf = self.info()
        shape = (inf.L[2] // 2 + 1, inf.L[1] // 2 + 1, inf.L[0] // 2 + 1)
        out = torch.empty(shape, dtype=self.torch_dtype, device="cuda")
        _check(_lib.ps_kernel_get(self._h, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out


def solve_batched(plans, rhos, Vs=None, energy=True, stream=None):
    """ps_solve_batched over a list of built plans and matching densities."""
    import torch
    lib = load_library()
    count = len(plans)
    if len(rhos) != count:
        raise ValueError("plans and rhos differ in length")
    for p, r in zip(plans, rhos):
        p._check_tensor(r, "rho")
    if Vs is None:
        Vs = [torch.empty_like(r) for r in rhos]
    E = torch.empty(count, dtype=torch.float64, device=rhos[0].device) if (energy and count) else None
    arr = ctypes.c_void_p * max(count, 1)
    hp = arr(*[p.handle for p in plans])
    rp = arr(*[r.data_ptr() for r in rhos])
    vp = arr(*[v.data_ptr() for v in Vs])
    _check(lib.ps_solve_batched(count, hp, rp, vp,
                                ctypes.c_void_p(E.data_ptr()) if E is not None else None,
                                _stream_handle(stream)))
    return Vs, E


def hartree_energy_noalloc(rho, V, h, E=None, stream=None):
    """ps_hartree_energy_noalloc: E = 1/2 h^3 sum rho V from device tensors,
    without any device allocation inside the library (``E``, a one-element
    float64 CUDA tensor, may be passed in so the call allocates nothing)."""
    import torch
    lib = load_library()
    if rho.shape != V.shape or rho.dtype != V.dtype or not (rho.is_cuda and V.is_cuda) \
            or not (rho.is_contiguous() and V.is_contiguous()):
        raise ValueError("rho and V must be contiguous CUDA tensors of one shape and dtype")
    dtype = {torch.float32: PS_F32, torch.float64: PS_F64}.get(rho.dtype)
    if dtype is None:
        raise ValueError("rho must be float32 or float64")
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=rho.device)
    _check(lib.ps_hartree_energy_noalloc(dtype, rho.numel(), float(h), ctypes.c_void_p(rho.data_ptr()),
                                         ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                         _stream_handle(stream)))
    return E
