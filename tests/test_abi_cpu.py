"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/wri.h declares, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import wri
    return wri


def test_exports_every_declared_symbol(W):
    hdr = open(os.path.join(ROOT, "include", "wri.h")).read()
    declared = set(re.findall(r"WRI_API\s+[\w\s\*]+?\b(wri_\w+)\s*\(", hdr))
    assert declared == set(W.EXPORTS)
    lib = C.CDLL(W.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_and_tiles(W):
    assert W.strerror(0) == "success"
    assert "invalid" in W.strerror(1)
    assert W.strerror(99) == "unknown error code"
    assert W.tile_shapes() == [(32, 4), (32, 8), (32, 16)]
    assert W.version().startswith("libwri")


class _FakeTensor:
    """Stands in for a device tensor: only its address is read by the marshalling."""

    def __init__(self, addr=0x10000):
        self.addr = addr

    def data_ptr(self):
        return self.addr


def _spec(W, **kw):
    base = dict(nx=20, ny=18, nz=16, npml=3, h=10.0, omega=60.0, v_max=2000.0, m=_FakeTensor(),
                src=np.array([1000, 1500]), rec_off=np.array([0, 3, 5]), rec_idx=np.array([10, 20, 30, 40, 50]),
                d=_FakeTensor(), lam=0.01, u=_FakeTensor())
    base.update(kw)
    return W.GroupSpec(**base)


def test_workspace_size_validation(W):
    o = W.make_opts()
    good = W.workspace_size([_spec(W)], o)
    assert good > 0
    n = 20 * 18 * 16
    # vectors r1 x2, p x2, s, t1 for 2 systems at 8 bytes per complex
    assert good >= 6 * 2 * n * 8
    assert W.aux_workspace_size([_spec(W)]) < good
    bad = [
        _spec(W, nx=2),
        _spec(W, npml=9),                               # 2*npml >= ny
        _spec(W, h=0.0),
        _spec(W, lam=-1.0),
        _spec(W, src=np.array([1000, n])),              # source out of range
        _spec(W, rec_idx=np.array([10, 20, 30, 40, n])),
        _spec(W, rec_idx=np.array([10, 20, 10, 40, 50])),  # duplicate receiver in system 0
        _spec(W, rec_off=np.array([1, 3, 5])),
        _spec(W, rec_off=np.array([0, 4, 3])),
        _spec(W, m=None),
    ]
    for s in bad:
        assert W.workspace_size([s], o) == 0
    assert W.workspace_size([_spec(W)], W.make_opts(dtype=7)) == 0
    assert W.workspace_size([_spec(W)], W.make_opts(max_iter=0)) == 0
    assert W.workspace_size([_spec(W)], W.make_opts(tol=float("nan"))) == 0
    assert W.workspace_size([_spec(W)] * 9, o) == 0        # more groups than one launch holds
    # refinement adds the FP64 master, the FP64 residual and the FP32 correction
    ir = W.workspace_size([_spec(W)], W.make_opts(max_refine=3))
    assert ir >= good + 2 * n * (8 + 16 + 16)
    assert W.workspace_size([_spec(W)], W.make_opts(max_refine=3, dtype=W.C128)) == 0


def test_direction_ring_in_the_workspace(W):
    """Configuration 24 (x updated every fourth iteration) keeps four search directions per system;
    the automatic kernel choice reserves them too, so that wri_autotune may pick it in a workspace
    sized before tuning. The other configurations, and batches the TMA phases cannot take, keep two.
    Kernel indices past the last configuration are rejected."""
    n = 20 * 18 * 16
    vec = 2 * n * 8  # one complex64 vector of the 2 systems (a multiple of the 256-byte alignment)

    def size(spec, kernel):
        return W.workspace_size([spec], W.make_opts(kernel=kernel))

    auto, quad, single, pair = (size(_spec(W), k) for k in (0, W.KERNEL_TMA(24), W.KERNEL_TMA(18), W.KERNEL_TMA(22)))
    assert single > 0 and pair == single
    assert auto == quad == single + 2 * vec
    odd = _spec(W, nx=22)  # x extent not a multiple of 4: z-march kernels whatever the request
    assert size(odd, 0) == size(odd, W.KERNEL_TMA(24)) > 0
    assert size(_spec(W), W.KERNEL_TMA(24) + 1) == 0


def test_solve_rejects_before_device_work(W):
    o = W.make_opts()
    m = W._Marshal([_spec(W, rec_idx=np.array([10, 20, 10, 40, 50]))])
    rc = W.lib.wri_solve_batch(m.arr, m.n, C.byref(o), 0x100, 0x200, 0x300, 0x1000, 1 << 30, None)
    assert rc == W.EINVAL
    m = W._Marshal([_spec(W)])
    # misaligned / too small workspace
    rc = W.lib.wri_solve_batch(m.arr, m.n, C.byref(o), 0x100, 0x200, 0x300, 0x1001, 1 << 30, None)
    assert rc == W.EWORKSPACE
    rc = W.lib.wri_solve_batch(m.arr, m.n, C.byref(o), 0x100, 0x200, 0x300, 0x1000, 16, None)
    assert rc == W.EWORKSPACE
    rc = W.lib.wri_solve_batch(m.arr, m.n, C.byref(o), None, 0x200, 0x300, 0x1000, 1 << 30, None)
    assert rc == W.EINVAL
    # refinement is C64 only; the baseline path does not refine
    o2 = W.make_opts(max_refine=2, plain=True)
    rc = W.lib.wri_solve_batch(m.arr, m.n, C.byref(o2), 0x100, 0x200, 0x300, 0x1000, 1 << 40, None)
    assert rc == W.ENOTSUP


def test_apply_rejects_overlap_and_bad_grid(W):
    g = W.WriGrid(20, 18, 16, 3, 10.0, 60.0, 1e-3, 2000.0)
    n = 20 * 18 * 16
    assert W.lib.wri_apply_A(C.byref(g), 0, 0x1000, 1, 0x100000, 0x100000 + 8 * (n - 1), None) == W.EINVAL
    g2 = W.WriGrid(20, 18, 16, 3, 10.0, 60.0, 2.0, 2000.0)   # pml_R outside (0, 1)
    assert W.lib.wri_apply_A(C.byref(g2), 0, 0x1000, 1, 0x100000, 0x900000, None) == W.EINVAL
    assert W.lib.wri_apply_AH(C.byref(g), 5, 0x1000, 1, 0x100000, 0x900000, None) == W.EINVAL


def test_autotune_validates_and_skips_unsupported_batches(W):
    """Argument errors come back before any device work; batches the TMA phases cannot take
    (complex128, the baseline path, the z-march kernels) return unchanged without touching the
    device.  (Refined batches are tuned: their inner solves run on the TMA phases.)"""
    m = W._Marshal([_spec(W)])
    o = W.make_opts()
    assert W.lib.wri_autotune(m.arr, m.n, C.byref(o), 1, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_autotune(m.arr, m.n, None, 8, 0x1000, 1 << 30, None) == W.EINVAL
    bad = W._Marshal([_spec(W, nx=2)])
    assert W.lib.wri_autotune(bad.arr, bad.n, C.byref(o), 8, 0x1000, 1 << 30, None) == W.EINVAL
    for kw in (dict(wait_limit_us=-1), dict(test_withhold=-2)):
        assert W.lib.wri_autotune(m.arr, m.n, C.byref(W.make_opts(**kw)), 8, 0x1000, 1 << 30, None) == W.EINVAL
        assert W.lib.wri_solve_batch(m.arr, m.n, C.byref(W.make_opts(**kw)), 0x100, 0x200, 0x300, 0x1000, 1 << 40,
                                     None) == W.EINVAL
    for kw in (dict(dtype=W.C128), dict(plain=True), dict(kernel=W.KERNEL_MARCH)):
        o2 = W.make_opts(**kw)
        before = bytes(o2)
        assert W.lib.wri_autotune(m.arr, m.n, C.byref(o2), 8, 0x1000, 1 << 30, None) == W.OK
        assert bytes(o2) == before


def test_fp64_wavefield_must_be_on_every_group_and_aligned(W):
    """u64 on some groups only, or misaligned, is rejected before any device work."""
    g1, g2 = _spec(W), _spec(W)
    g2.u64 = _FakeTensor(0x20000)
    m = W._Marshal([g1, g2])
    gp = (C.c_void_p * 2)(0x4000, 0x5000)
    assert W.lib.wri_gradient(m.arr, 2, W.C64, 0x3000, gp, 0x6000, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_source_estimate(m.arr, 2, W.C64, 0x3000, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_gradient_noalloc(m.arr, 2, W.C64, 0x3000, gp, 0x6000, None) == W.EINVAL
    g1.u64 = _FakeTensor(0x20008)  # both set, one not 16-byte aligned
    m = W._Marshal([g1, g2])
    assert W.lib.wri_source_estimate(m.arr, 2, W.C64, 0x3000, 0x1000, 1 << 30, None) == W.EINVAL
    o = W.make_opts()
    assert W.lib.wri_solve_batch(m.arr, 2, C.byref(o), 0x100, 0x200, 0x300, 0x1000, 1 << 40, None) == W.EINVAL


def test_gradient_refined_needs_a_refined_solve_of_the_same_problem(W):
    """wri_gradient_refined: no refinement in the options, no FP64 wavefield, or a workspace that holds
    no residual of this problem are argument errors, caught before any device work."""
    g = _spec(W, u64=_FakeTensor(0x20000))
    m = W._Marshal([g])
    gp = (C.c_void_p * 1)(0x4000)
    ref = W.make_opts(max_refine=1)
    assert W.lib.wri_gradient_refined(m.arr, 1, C.byref(ref), gp, 0x6000, 0x100000, 1 << 40, None) == W.EINVAL
    assert W.lib.wri_gradient_refined(m.arr, 1, C.byref(W.make_opts()), gp, 0x6000, 0x100000, 1 << 40,
                                      None) == W.EINVAL
    m2 = W._Marshal([_spec(W)])
    assert W.lib.wri_gradient_refined(m2.arr, 1, C.byref(ref), gp, 0x6000, 0x100000, 1 << 40, None) == W.EINVAL


def test_general_right_hand_side_and_fwi_calls_validate(W):
    """lambda = 0 needs a known right-hand side (alpha or q), alpha and q together are an error, and
    the reduced-FWI calls reject missing outputs before any device work."""
    o = W.make_opts()
    assert W.workspace_size([_spec(W, lam=0.0)], o) == 0                               # source-free, no data
    assert W.workspace_size([_spec(W, lam=0.0, q=_FakeTensor(0x30000))], o) > 0
    assert W.workspace_size([_spec(W, lam=0.0, alpha=_FakeTensor(0x30000))], o) > 0
    assert W.workspace_size([_spec(W, alpha=_FakeTensor(0x30000), q=_FakeTensor(0x40000))], o) == 0
    m = W._Marshal([_spec(W)])
    qp = (C.c_void_p * 1)(0x5000)
    assert W.lib.wri_fwi_adjoint_source(m.arr, 1, 0, None, None, qp, 0x6000, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_fwi_adjoint_source(m.arr, 1, 7, None, 0x7000, qp, 0x6000, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_fwi_adjoint_source(m.arr, 1, 0, None, 0x7000, qp, 0x6000, 0x1001, 1 << 30, None) == W.EWORKSPACE
    gp = (C.c_void_p * 1)(0x8000)
    assert W.lib.wri_fwi_gradient(m.arr, 1, 0, None, qp, gp, None) == W.EINVAL
    assert W.lib.wri_fwi_gradient(m.arr, 1, 0, 0x9000, (C.c_void_p * 1)(None), gp, None) == W.EINVAL


def test_tv_rejects_invalid_arguments(W):
    g = W.WriGrid(20, 18, 16, 3, 10.0, 60.0, 1e-3, 2000.0)
    assert W.lib.wri_tv(C.byref(g), 0x1000, 0.0, 1.0, 0x2000, None, None) == W.EINVAL      # beta = 0
    assert W.lib.wri_tv(C.byref(g), 0x1000, 0.1, -1.0, 0x2000, None, None) == W.EINVAL     # gamma < 0
    assert W.lib.wri_tv(C.byref(g), None, 0.1, 1.0, 0x2000, None, None) == W.EINVAL        # no model
    assert W.lib.wri_tv(C.byref(g), 0x1000, 0.1, 1.0, None, None, None) == W.EINVAL        # no output
    g2 = W.WriGrid(2, 18, 16, 0, 10.0, 60.0, 1e-3, 2000.0)
    assert W.lib.wri_tv(C.byref(g2), 0x1000, 0.1, 1.0, 0x2000, None, None) == W.EINVAL


def test_empty_batches_are_rejected(W):
    """A group without systems, a call without groups and a NULL group array are argument errors
    (nsys >= 1 and at least one group), caught before any device work."""
    o = W.make_opts()
    empty = _spec(W, src=np.zeros(0, np.int64), rec_off=np.array([0], np.int32), rec_idx=np.zeros(0, np.int32))
    assert W.workspace_size([empty], o) == 0
    assert W.workspace_size([_spec(W), empty], o) == 0
    m = W._Marshal([_spec(W)])
    assert W.lib.wri_workspace_size(m.arr, 0, C.byref(o)) == 0
    assert W.lib.wri_solve_batch(m.arr, 0, C.byref(o), 0x100, 0x200, 0x300, 0x1000, 1 << 30, None) == W.EINVAL
    assert W.lib.wri_solve_batch(None, 1, C.byref(o), 0x100, 0x200, 0x300, 0x1000, 1 << 30, None) == W.EINVAL


def test_binding_rejects_host_and_mismatched_tensors(W, monkeypatch):
    """Tensors handed to the library as device pointers are checked before any library call:
    contiguous, of the call's dtype, large enough, and on a CUDA device.  A host tensor would
    otherwise reach the kernels as a bad device address."""
    import torch

    class NoLib:
        def __getattr__(self, name):
            raise AssertionError(f"{name} called although the arguments are invalid")

    n = 20 * 18 * 16
    with pytest.raises(ValueError, match="contiguous"):
        W._device_tensor(torch.zeros(4, 4).t(), "x")
    with pytest.raises(ValueError, match="float64"):
        W._device_tensor(torch.zeros(4, dtype=torch.float32), "m", None, torch.float64, 4)
    with pytest.raises(ValueError, match="elements"):
        W._device_tensor(torch.zeros(3, dtype=torch.float64), "m", None, torch.float64, 4)
    with pytest.raises(ValueError, match="CUDA"):
        W._device_tensor(torch.zeros(4, dtype=torch.float64), "m", None, torch.float64, 4)
    assert W._device_tensor(_FakeTensor(), "m", "dev0") == "dev0"          # pointer holders pass through

    host = _spec(W, m=torch.zeros(16, 18, 20), d=torch.zeros(5, dtype=torch.complex64),
                 u=torch.zeros(2, n, dtype=torch.complex64))
    with pytest.raises(ValueError, match="group 0: m must be a CUDA tensor"):
        W._Marshal([host], W.C64)
    with pytest.raises(ValueError, match="group 0: m must be torch.float64"):
        W._Marshal([host], W.C128)
    with pytest.raises(ValueError, match="group 0: u holds"):
        W._Marshal([_spec(W, u=torch.zeros(1, n, dtype=torch.complex64))], W.C64)
    monkeypatch.setattr(W, "lib", NoLib())
    with pytest.raises(ValueError):
        W.solve([host], W.make_opts())
    with pytest.raises(ValueError):
        W.apply_A(_spec(W, m=torch.zeros(16, 18, 20)), torch.zeros(2, n, dtype=torch.complex64))
    with pytest.raises(ValueError):
        W.tv(_spec(W), torch.zeros(16, 18, 20, dtype=torch.float64), 0.1)
    with pytest.raises(ValueError, match="gradient buffers"):
        W.gradient_noalloc([_spec(W)], W.C64, torch.zeros(2, dtype=torch.complex128), [], torch.zeros(1))
