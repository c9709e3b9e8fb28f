"""ctypes binding of libwri (include/wri.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of ``libwri.so``.  Tensors are
PyTorch CUDA tensors (device memory and streams); geometry (source and receiver
node indices) is host numpy data.  If the shared library is missing this module
raises at import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwri.so")

OK, EINVAL, ECUDA, EWORKSPACE, ENOTSUP, ESCRATCH = 0, 1, 2, 3, 4, 5
NOALLOC_SCRATCH_BYTES = 4 << 20
SYS_OK, SYS_MAXITER, SYS_BREAKDOWN, SYS_NONFINITE = 0, 1, 2, 3
C64, C128 = 0, 1


class WriGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("npml", C.c_int32),
                ("h", C.c_double), ("omega", C.c_double), ("pml_R", C.c_double), ("v_max", C.c_double)]


class WriGroup(C.Structure):
    _fields_ = [("grid", WriGrid), ("m", C.c_void_p), ("nsys", C.c_int32), ("src_idx", C.c_void_p),
                ("rec_off", C.c_void_p), ("rec_idx", C.c_void_p), ("d", C.c_void_p), ("alpha", C.c_void_p),
                ("lam", C.c_double), ("u", C.c_void_p), ("u64", C.c_void_p), ("q", C.c_void_p)]


class WriSolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("dtype", C.c_int32),
                ("warm_start", C.c_int32), ("max_refine", C.c_int32), ("refine_tol", C.c_double),
                ("inner_tol", C.c_double), ("plain", C.c_int32), ("poll_every", C.c_int32),
                ("tile", C.c_int32), ("zsplit", C.c_int32), ("kernel", C.c_int32), ("order", C.c_int32),
                ("l2_promotion", C.c_int32), ("wait_limit_us", C.c_int32), ("host_loop", C.c_int32),
                ("test_withhold", C.c_int32)]


class WriError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} (code {code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libwri.so not built ({LIB_PATH}); run python -m paper_2410_18429_gb300.build")
    lib = C.CDLL(LIB_PATH)
    vp, i32, sz, dp = C.c_void_p, C.c_int, C.c_size_t, C.c_void_p
    lib.wri_apply_A.argtypes = [C.POINTER(WriGrid), i32, vp, i32, vp, vp, vp]
    lib.wri_apply_AH.argtypes = [C.POINTER(WriGrid), i32, vp, i32, vp, vp, vp]
    lib.wri_workspace_size.argtypes = [C.POINTER(WriGroup), i32, C.POINTER(WriSolveOpts)]
    lib.wri_workspace_size.restype = sz
    lib.wri_aux_workspace_size.argtypes = [C.POINTER(WriGroup), i32]
    lib.wri_aux_workspace_size.restype = sz
    lib.wri_solve_batch.argtypes = [C.POINTER(WriGroup), i32, C.POINTER(WriSolveOpts), vp, vp, vp, vp, sz, vp]
    lib.wri_source_estimate.argtypes = [C.POINTER(WriGroup), i32, i32, dp, vp, sz, vp]
    lib.wri_gradient.argtypes = [C.POINTER(WriGroup), i32, i32, dp, C.POINTER(C.c_void_p), dp, vp, sz, vp]
    lib.wri_gradient_noalloc.argtypes = [C.POINTER(WriGroup), i32, i32, dp, C.POINTER(C.c_void_p), dp, vp]
    lib.wri_gradient_refined.argtypes = [C.POINTER(WriGroup), i32, C.POINTER(WriSolveOpts), C.POINTER(C.c_void_p), dp,
                                         vp, sz, vp]
    lib.wri_autotune.argtypes = [C.POINTER(WriGroup), i32, C.POINTER(WriSolveOpts), i32, vp, sz, vp]
    lib.wri_fwi_adjoint_source.argtypes = [C.POINTER(WriGroup), i32, i32, dp, dp, C.POINTER(C.c_void_p), dp, vp, sz,
                                           vp]
    lib.wri_fwi_gradient.argtypes = [C.POINTER(WriGroup), i32, i32, dp, C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), vp]
    lib.wri_tv.argtypes = [C.POINTER(WriGrid), dp, C.c_double, C.c_double, dp, dp, vp]
    lib.wri_tile_count.argtypes = []
    lib.wri_tile_shape.argtypes = [i32, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.wri_strerror.argtypes = [i32]
    lib.wri_strerror.restype = C.c_char_p
    lib.wri_version.restype = C.c_char_p
    for f in ("wri_apply_A", "wri_apply_AH", "wri_solve_batch", "wri_source_estimate", "wri_gradient",
              "wri_gradient_noalloc", "wri_gradient_refined", "wri_fwi_adjoint_source", "wri_fwi_gradient",
              "wri_autotune", "wri_tv", "wri_tile_count", "wri_tile_shape"):
        getattr(lib, f).restype = C.c_int
    return lib


lib = _load()

EXPORTS = ("wri_apply_A", "wri_apply_AH", "wri_workspace_size", "wri_aux_workspace_size", "wri_solve_batch",
           "wri_source_estimate", "wri_gradient", "wri_gradient_noalloc", "wri_gradient_refined",
           "wri_fwi_adjoint_source", "wri_fwi_gradient", "wri_autotune", "wri_tv", "wri_tile_count",
           "wri_tile_shape", "wri_strerror", "wri_version")


def strerror(code: int) -> str:
    return lib.wri_strerror(int(code)).decode()


def version() -> str:
    return lib.wri_version().decode()


def _check(code: int, what: str):
    if code != OK:
        raise WriError(code, what)


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


@dataclass
class GroupSpec:
    """One frequency group: grid, model and systems (see ``wri_group`` in include/wri.h).

    m: real CUDA tensor [nz, ny, nx] (float32 for C64, float64 for C128);
    src: int64 [nsys]; rec_off: int32 [nsys+1]; rec_idx: int32 [nnz] (host numpy);
    d: complex CUDA tensor [nnz]; alpha: float64 CUDA tensor [nsys, 2] or None (source-free);
    u: complex CUDA tensor [nsys, n] (initial guess with warm_start, result on return).
    u64: optional complex128 CUDA tensor [nsys, n] for complex64 problems: the solve also writes
    the FP64 solution there, and the source estimate and gradient then read it (FP64 stencils).
    q: optional complex CUDA tensor [nsys, n] (dtype of u): a general PDE right-hand side b1 = q in
    place of alpha e (alpha must then be None); lam may be 0 when alpha or q is given.
    """

    nx: int
    ny: int
    nz: int
    npml: int
    h: float
    omega: float
    v_max: float
    m: object
    src: np.ndarray
    rec_off: np.ndarray
    rec_idx: np.ndarray
    d: object
    lam: float
    u: object
    alpha: object = None
    pml_R: float = 1e-3
    u64: object = None
    q: object = None

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nsys(self) -> int:
        return len(self.src)

    def grid(self) -> WriGrid:
        return WriGrid(self.nx, self.ny, self.nz, self.npml, self.h, self.omega, self.pml_R, self.v_max)


def _device_tensor(t, what: str, dev=None, dtype=None, min_numel: Optional[int] = None):
    """Check a tensor handed to the library as a device pointer: on a CUDA device (the same as
    the call's other tensors), contiguous, of the dtype the call's arithmetic reads and large
    enough.  A host tensor or a short buffer would otherwise reach the kernels as a bad device
    address.  Objects that are not torch tensors (raw pointer holders) are passed through: the
    library checks what it can.  Returns the device seen so far."""
    import torch
    if not isinstance(t, torch.Tensor):
        return dev
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype} for this call (it is {t.dtype})")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{what} holds {t.numel()} elements; {min_numel} are needed")
    if t.device.type != "cuda":
        raise ValueError(f"{what} must be a CUDA tensor (it is on {t.device})")
    if dev is not None and t.device != dev:
        raise ValueError(f"{what} is on {t.device}, the call's other tensors on {dev}")
    return t.device


def _dtypes(dtype):
    """(real, complex) torch dtypes of the arithmetic type ``dtype`` (None: not known here)."""
    import torch
    if dtype == C64:
        return torch.float32, torch.complex64
    if dtype == C128:
        return torch.float64, torch.complex128
    return None, None


class _Marshal:
    """Builds the C array of wri_group and keeps the host geometry alive.  With the call's
    arithmetic type ``dtype`` the groups' tensors are checked against it (``_device_tensor``)."""

    def __init__(self, groups: Sequence[GroupSpec], dtype: Optional[int] = None):
        import torch
        self.keep = []
        arr = (WriGroup * len(groups))()
        real, cplx = _dtypes(dtype)
        dev = None
        for i, g in enumerate(groups):
            src = np.ascontiguousarray(g.src, dtype=np.int64)
            off = np.ascontiguousarray(g.rec_off, dtype=np.int32)
            rec = np.ascontiguousarray(g.rec_idx, dtype=np.int32)
            nsys, n = len(src), g.nx * g.ny * g.nz
            nnz = int(off[-1]) if len(off) else 0
            dev = _device_tensor(g.m, f"group {i}: m", dev, real, n)
            dev = _device_tensor(g.d, f"group {i}: d", dev, cplx, nnz)
            dev = _device_tensor(g.u, f"group {i}: u", dev, cplx, nsys * n)
            dev = _device_tensor(g.alpha, f"group {i}: alpha", dev, torch.float64, 2 * nsys)
            dev = _device_tensor(g.u64, f"group {i}: u64", dev, torch.complex128, nsys * n)
            dev = _device_tensor(g.q, f"group {i}: q", dev, cplx, nsys * n)
            if len(rec) == 0:
                rec = np.zeros(1, dtype=np.int32)
            self.keep += [src, off, rec]
            arr[i] = WriGroup(g.grid(), _ptr(g.m), len(src), src.ctypes.data, off.ctypes.data, rec.ctypes.data,
                              _ptr(g.d), _ptr(g.alpha), float(g.lam), _ptr(g.u), _ptr(g.u64), _ptr(g.q))
        self.arr = arr
        self.n = len(groups)
        self.device = dev


KERNEL_AUTO, KERNEL_MARCH = 0, 1


def KERNEL_TMA(cfg: int = 0) -> int:
    return 2 + int(cfg)


def make_opts(tol=1e-6, max_iter=10000, dtype=C64, warm_start=False, max_refine=0, refine_tol=1e-10,
              inner_tol=1e-3, plain=False, poll_every=0, tile=0, zsplit=0, kernel=KERNEL_AUTO,
              order=0, l2_promotion=0, wait_limit_us=0, host_loop=False, test_withhold=0) -> WriSolveOpts:
    return WriSolveOpts(float(tol), int(max_iter), int(dtype), int(bool(warm_start)), int(max_refine),
                        float(refine_tol), float(inner_tol), int(bool(plain)), int(poll_every), int(tile),
                        int(zsplit), int(kernel), int(order), int(l2_promotion), int(wait_limit_us),
                        int(bool(host_loop)), int(test_withhold))


def workspace_size(groups: Sequence[GroupSpec], opts: WriSolveOpts) -> int:
    m = _Marshal(groups, int(opts.dtype))
    return int(lib.wri_workspace_size(m.arr, m.n, C.byref(opts)))


def aux_workspace_size(groups: Sequence[GroupSpec]) -> int:
    m = _Marshal(groups)
    return int(lib.wri_aux_workspace_size(m.arr, m.n))


def _workspace(nbytes: int, device, workspace=None):
    import torch
    if workspace is not None and workspace.numel() >= nbytes:
        _device_tensor(workspace, "workspace", device if isinstance(device, torch.device) and
                       device.type == "cuda" else None)
        return workspace
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def apply_A(g: GroupSpec, x, adjoint: bool = False, out=None, stream=None):
    """y = A x (or A^H x) for x [nsys, n] complex on the device."""
    import torch
    dtype = C128 if x.dtype == torch.complex128 else C64
    y = torch.empty_like(x) if out is None else out
    grid = g.grid()
    nsys = x.shape[0] if x.dim() > 1 else 1
    real, cplx = _dtypes(dtype)
    dev = _device_tensor(x, "x", None, cplx, nsys * g.n)
    dev = _device_tensor(y, "out", dev, cplx, nsys * g.n)
    _device_tensor(g.m, "m", dev, real, g.n)
    f = lib.wri_apply_AH if adjoint else lib.wri_apply_A
    _check(f(C.byref(grid), dtype, _ptr(g.m), nsys, _ptr(x), _ptr(y), _stream(stream)), "wri_apply_A")
    return y


def solve(groups: Sequence[GroupSpec], opts: WriSolveOpts, workspace=None, stream=None):
    """Solve every system; returns (iters int32, relres float64, status int32) CUDA tensors."""
    import torch
    m = _Marshal(groups, int(opts.dtype))
    dev = groups[0].u.device
    nsys = sum(g.nsys for g in groups)
    nbytes = lib.wri_workspace_size(m.arr, m.n, C.byref(opts))
    if nbytes == 0:
        raise WriError(EINVAL, "wri_workspace_size")
    ws = _workspace(nbytes, dev, workspace)
    iters = torch.zeros(nsys, dtype=torch.int32, device=dev)
    relres = torch.zeros(nsys, dtype=torch.float64, device=dev)
    status = torch.zeros(nsys, dtype=torch.int32, device=dev)
    _check(lib.wri_solve_batch(m.arr, m.n, C.byref(opts), _ptr(iters), _ptr(relres), _ptr(status), _ptr(ws),
                               ws.numel(), _stream(stream)), "wri_solve_batch")
    return iters, relres, status


def source_estimate(groups: Sequence[GroupSpec], dtype: int, workspace=None, stream=None):
    """a_i = (A u_i)[src_i] for every system; returns complex128 CUDA tensor [sum nsys]."""
    import torch
    m = _Marshal(groups, dtype)
    dev = groups[0].u.device
    nsys = sum(g.nsys for g in groups)
    ws = _workspace(lib.wri_aux_workspace_size(m.arr, m.n), dev, workspace)
    out = torch.zeros(nsys, 2, dtype=torch.float64, device=dev)
    _check(lib.wri_source_estimate(m.arr, m.n, dtype, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
           "wri_source_estimate")
    return torch.view_as_complex(out)


def _check_outputs(groups, a, grads, f, dev):
    """The weights read and the gradient and objective buffers written by a gradient call."""
    import torch
    if len(grads) != len(groups):
        raise ValueError(f"{len(grads)} gradient buffers for {len(groups)} groups")
    dev = _device_tensor(a, "alpha", dev, torch.float64, 2 * sum(g.nsys for g in groups))
    for i, (g, t) in enumerate(zip(groups, grads)):
        dev = _device_tensor(t, f"gradient {i}", dev, torch.float64, g.n)
    _device_tensor(f, "f", dev, torch.float64, 1)


def gradient(groups: Sequence[GroupSpec], dtype: int, alpha, grads=None, f=None, workspace=None, stream=None):
    """Accumulate g and f (Eqs. VarG2 / VarObj2).  alpha: complex128 [sum nsys].

    Returns (list of float64 gradient tensors shaped like each group's m, f tensor [1])."""
    import torch
    m = _Marshal(groups, dtype)
    dev = groups[0].u.device
    ws = _workspace(lib.wri_aux_workspace_size(m.arr, m.n), dev, workspace)
    if grads is None:
        grads = [torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64, device=dev) for g in groups]
    if f is None:
        f = torch.zeros(1, dtype=torch.float64, device=dev)
    a = torch.view_as_real(alpha.to(torch.complex128).contiguous())
    _check_outputs(groups, a, grads, f, m.device)
    gp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in grads])
    _check(lib.wri_gradient(m.arr, m.n, dtype, _ptr(a), gp, _ptr(f), _ptr(ws), ws.numel(), _stream(stream)),
           "wri_gradient")
    return grads, f


def gradient_refined(groups: Sequence[GroupSpec], opts: WriSolveOpts, workspace, grads=None, f=None, stream=None):
    """wri_gradient_refined: g and f from the FP64 residual a refined solve left in ``workspace``.

    Call after ``solve(groups, opts, workspace=workspace)`` with max_refine > 0 and u64 on every
    group, with the same groups, options and workspace.  Returns (gradients, f) like gradient()."""
    import torch
    m = _Marshal(groups, int(opts.dtype))
    dev = groups[0].u.device
    if grads is None:
        grads = [torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64, device=dev) for g in groups]
    if f is None:
        f = torch.zeros(1, dtype=torch.float64, device=dev)
    if len(grads) != len(groups):
        raise ValueError(f"{len(grads)} gradient buffers for {len(groups)} groups")
    for i, (g, t) in enumerate(zip(groups, grads)):
        _device_tensor(t, f"gradient {i}", m.device, torch.float64, g.n)
    _device_tensor(f, "f", m.device, torch.float64, 1)
    _device_tensor(workspace, "workspace", m.device)
    gp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in grads])
    _check(lib.wri_gradient_refined(m.arr, m.n, C.byref(opts), gp, _ptr(f), _ptr(workspace), workspace.numel(),
                                    _stream(stream)), "wri_gradient_refined")
    return grads, f


def fwi_adjoint_source(groups: Sequence[GroupSpec], dtype: int, q_adj, alpha=None, f=None, workspace=None,
                       stream=None):
    """wri_fwi_adjoint_source: weights (given ``alpha`` or source-free estimates), f += 1/2 sum ||r||^2
    and the adjoint right-hand sides conj(P^T r) written into ``q_adj`` (one zeroed tensor [nsys, n]
    per group) from the forward wavefields G in ``groups[g].u``.  Returns (weights complex128 [sum
    nsys], f tensor [1])."""
    import torch
    m = _Marshal(groups, dtype)
    dev = groups[0].u.device
    nsys = sum(g.nsys for g in groups)
    _, cplx = _dtypes(dtype)
    if len(q_adj) != len(groups):
        raise ValueError(f"{len(q_adj)} adjoint right-hand sides for {len(groups)} groups")
    for i, (g, t) in enumerate(zip(groups, q_adj)):
        _device_tensor(t, f"q_adj {i}", m.device, cplx, g.nsys * g.n)
    a_in = None
    if alpha is not None:
        a_in = torch.view_as_real(alpha.to(torch.complex128).contiguous())
        _device_tensor(a_in, "alpha", m.device, torch.float64, 2 * nsys)
    a_out = torch.zeros(nsys, 2, dtype=torch.float64, device=dev)
    if f is None:
        f = torch.zeros(1, dtype=torch.float64, device=dev)
    _device_tensor(f, "f", m.device, torch.float64, 1)
    ws = _workspace(lib.wri_aux_workspace_size(m.arr, m.n), dev, workspace)
    qp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in q_adj])
    _check(lib.wri_fwi_adjoint_source(m.arr, m.n, dtype, _ptr(a_in), _ptr(a_out), qp, _ptr(f), _ptr(ws), ws.numel(),
                                      _stream(stream)), "wri_fwi_adjoint_source")
    return torch.view_as_complex(a_out), f


def fwi_gradient(groups: Sequence[GroupSpec], dtype: int, alpha, w_adj, grads=None, stream=None):
    """wri_fwi_gradient: grad += -omega^2 sum Re(w a G w_adj) from the forward wavefields G
    (``groups[g].u``), the weights and the adjoint solves' wavefields ``w_adj``."""
    import torch
    m = _Marshal(groups, dtype)
    dev = groups[0].u.device
    _, cplx = _dtypes(dtype)
    if grads is None:
        grads = [torch.zeros(g.nz, g.ny, g.nx, dtype=torch.float64, device=dev) for g in groups]
    a = torch.view_as_real(alpha.to(torch.complex128).contiguous())
    _device_tensor(a, "alpha", m.device, torch.float64, 2 * sum(g.nsys for g in groups))
    for i, (g, t, w) in enumerate(zip(groups, grads, w_adj)):
        _device_tensor(t, f"gradient {i}", m.device, torch.float64, g.n)
        _device_tensor(w, f"w_adj {i}", m.device, cplx, g.nsys * g.n)
    wp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in w_adj])
    gp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in grads])
    _check(lib.wri_fwi_gradient(m.arr, m.n, dtype, _ptr(a), wp, gp, _stream(stream)), "wri_fwi_gradient")
    return grads


def gradient_noalloc(groups: Sequence[GroupSpec], dtype: int, alpha, grads, f, stream=None):
    """wri_gradient_noalloc: like gradient() but without a workspace (static device scratch).

    For callers that cannot allocate device memory; grads and f are caller-owned
    tensors that are accumulated into."""
    import torch
    m = _Marshal(groups, dtype)
    a = torch.view_as_real(alpha.to(torch.complex128).contiguous())
    _check_outputs(groups, a, grads, f, m.device)
    gp = (C.c_void_p * len(groups))(*[t.data_ptr() for t in grads])
    _check(lib.wri_gradient_noalloc(m.arr, m.n, dtype, _ptr(a), gp, _ptr(f), _stream(stream)),
           "wri_gradient_noalloc")
    return grads, f


def _tune_key(groups: Sequence[GroupSpec], opts: WriSolveOpts, device) -> str:
    """What the autotuner's choice depends on: the GPU, the library build (its version string
    carries the kernel-source hash), the options that shape the solve, and every group's grid,
    system count, receiver count and mode."""
    import torch
    name = torch.cuda.get_device_name(device) if device.type == "cuda" else device.type
    parts = [name, version(), f"dtype={opts.dtype} refine={opts.max_refine} plain={opts.plain} tile={opts.tile} "
             f"zsplit={opts.zsplit} l2={opts.l2_promotion}"]
    for g in groups:
        parts.append(f"{g.nx}x{g.ny}x{g.nz}+{g.npml} nsys={g.nsys} nnz={len(g.rec_idx)} "
                     f"{'free' if g.alpha is None else 'known'}")
    return " | ".join(parts)


def _read_tune_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            table = json.load(fh)
        return table if isinstance(table, dict) else {}
    except (OSError, ValueError):
        return {}


def autotune(groups: Sequence[GroupSpec], opts: WriSolveOpts, trial_iters: int = 12, workspace=None, stream=None,
             cache: Optional[str] = None):
    """wri_autotune: a copy of opts with the fastest (kernel, order) for this batch.

    The groups' wavefields are overwritten by the trial solves (unless the choice is cached).
    ``cache``: a JSON file that keeps choices across processes (default: the file named by the
    environment variable WRI_TUNE_CACHE, else none).  A choice stored there for the same GPU,
    library build, options and batch shape is reused without trial solves; a missing or
    unreadable file counts as empty, and new choices are written to a temporary file that then
    replaces it."""
    path = cache if cache is not None else os.environ.get("WRI_TUNE_CACHE")
    dev = groups[0].u.device
    key = _tune_key(groups, opts, dev) if path else None
    if path:
        hit = _read_tune_cache(path).get(key)
        if isinstance(hit, dict) and "kernel" in hit and "order" in hit:
            out = WriSolveOpts.from_buffer_copy(opts)
            out.kernel, out.order = int(hit["kernel"]), int(hit["order"])
            return out
    m = _Marshal(groups, int(opts.dtype))
    nbytes = lib.wri_workspace_size(m.arr, m.n, C.byref(opts))
    if nbytes == 0:
        raise WriError(EINVAL, "wri_workspace_size")
    ws = _workspace(nbytes, dev, workspace)
    out = WriSolveOpts.from_buffer_copy(opts)
    _check(lib.wri_autotune(m.arr, m.n, C.byref(out), int(trial_iters), _ptr(ws), ws.numel(), _stream(stream)),
           "wri_autotune")
    if path:
        table = _read_tune_cache(path)
        table[key] = {"kernel": int(out.kernel), "order": int(out.order)}
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return out


def tv(g: GroupSpec, m, beta: float, gamma: float = 1.0, out=None, grad=None, stream=None):
    """wri_tv: (tv [1] float64, grad) with tv += gamma TV(m) and grad += gamma dTV/dm (if given).

    m: float64 CUDA tensor shaped like the group's grid."""
    import torch
    mm = m.detach().to(torch.float64).contiguous()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=mm.device)
    dev = _device_tensor(mm, "m", None, torch.float64, g.n)
    dev = _device_tensor(out, "tv", dev, torch.float64, 1)
    _device_tensor(grad, "grad", dev, torch.float64, g.n)
    grid = g.grid()
    _check(lib.wri_tv(C.byref(grid), _ptr(mm), float(beta), float(gamma), _ptr(out), _ptr(grad), _stream(stream)),
           "wri_tv")
    return out, grad


def tile_shapes():
    out = []
    for t in range(1, lib.wri_tile_count() + 1):
        bx, by = C.c_int(), C.c_int()
        _check(lib.wri_tile_shape(t, C.byref(bx), C.byref(by)), "wri_tile_shape")
        out.append((bx.value, by.value))
    return out
