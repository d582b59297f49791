"""C-ABI checks that need no GPU: the library builds and loads, exports every symbol the
header declares, validates its arguments, and builds filters as documented."""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vkt.h")


def _device_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# The *_without_device tests hand the library fake device addresses and expect each call to
# stop at argument validation or at the device check.  Where a GPU is visible the device
# check passes and a kernel would run on those addresses, so they skip there.
without_device = pytest.mark.skipif(_device_visible(),
                                    reason="fake device pointers: only where no GPU is visible")


@pytest.fixture(scope="module")
def vkt():
    import paper_2203_10213_gb300 as m
    return m


@pytest.fixture(scope="module")
def lib(vkt):
    return vkt._lib


def test_exports_every_declared_symbol(lib):
    from paper_2203_10213_gb300._lib import SIGNATURES, declared_symbols
    names = declared_symbols(HEADER)
    assert len(names) >= 30
    for name in names:
        assert hasattr(lib, name), f"{name} declared in vkt.h but not exported"
        assert name in SIGNATURES, f"{name} has no Python binding"
    # and nothing beyond the vkt* API leaks out of the shared library
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True)
    if out.returncode == 0:
        exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
        assert {n for n in exported if n.startswith("vkt")} == set(names)


def test_error_strings(lib):
    for code in range(9):
        assert lib.vktGetErrorString(code)
    assert lib.vktGetErrorString(99) == b"unknown error"


def test_policy_roundtrip(vkt, lib):
    pol = vkt.ExecutionPolicy()
    pol.stream = None
    pol.printTimes = 1
    pol.debug = 0
    pol.path = vkt.PATH_DIRECT
    assert lib.vktSetThreadExecutionPolicy(pol) == 0
    got = vkt.ExecutionPolicy()
    assert lib.vktGetThreadExecutionPolicy(ctypes.byref(got)) == 0
    assert (got.printTimes, got.path) == (1, vkt.PATH_DIRECT)
    pol.path = 17
    assert lib.vktSetThreadExecutionPolicy(pol) == 1
    pol.path = 0
    pol.printTimes = 0
    assert lib.vktSetThreadExecutionPolicy(pol) == 0


@without_device
def test_volume_argument_validation(vkt, lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x10000)
    cv = lib.vktStructuredVolumeCreateView
    assert cv(None, fake, 4, 4, 4, vkt.F32, 1, 1, 1, 0, 1) == 1
    assert cv(ctypes.byref(h), None, 4, 4, 4, vkt.F32, 1, 1, 1, 0, 1) == 1
    assert cv(ctypes.byref(h), fake, 0, 4, 4, vkt.F32, 1, 1, 1, 0, 1) == 1
    assert cv(ctypes.byref(h), fake, 4, 4, 4, 7, 1, 1, 1, 0, 1) == 1
    assert cv(ctypes.byref(h), fake, 4, 4, 4, vkt.U8, 1, 1, 1, 0.5, 0.5) == 1   # lo == hi
    assert cv(ctypes.byref(h), fake, 4, 4, 4, vkt.F32, 0, 1, 1, 0, 1) == 1      # cell size
    assert cv(ctypes.byref(h), ctypes.c_void_p(0x10001), 4, 4, 4, vkt.F32, 1, 1, 1, 0, 1) == 1
    # a valid view needs no device: it only records the pointer
    assert cv(ctypes.byref(h), fake, 5, 6, 7, vkt.U16, 1, 2, 3, -1, 2) == 0
    v = vkt.StructuredVolume(h)
    assert v.dims == (5, 6, 7)
    assert v.format == vkt.U16
    assert v.cell_size == (1.0, 2.0, 3.0)
    assert v.mapping == (-1.0, 2.0)
    assert v.nbytes == 5 * 6 * 7 * 2
    assert v.data_ptr == 0x10000
    v.set_mapping(0.0, 4.0)
    assert v.mapping == (0.0, 4.0)
    with pytest.raises(vkt.VktError):
        v.set_mapping(1.0, 1.0)
    v.destroy()
    assert lib.vktStructuredVolumeDestroy(None) == 2


@without_device
def test_apply_filter_validation_without_device(vkt, lib):
    fake1, fake2 = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000)
    a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(a), fake1, 8, 8, 8, vkt.F32, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(b), fake2, 8, 8, 9, vkt.F32, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(c), ctypes.c_void_p(0x100100), 8, 8, 8,
                                             vkt.F32, 1, 1, 1, 0, 1) == 0
    f = vkt.Filter.gaussian(3, 1.0)
    assert lib.vktApplyFilterSV(None, a, f.handle) == 2
    assert lib.vktApplyFilterSV(a, b, f.handle) == 3          # dims mismatch
    assert lib.vktApplyFilterSV(a, c, f.handle) == 1          # overlapping memory
    for h in (a, b, c):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_backward_validation_without_device(vkt, lib):
    """vktApplyFilterBackwardSV and its allocation-free weight-gradient variant check their
    handles, formats, dims, aliasing and the gradient pointer before they need a device."""
    def view(addr, dims=(8, 8, 8), fmt=None):
        h = ctypes.c_void_p()
        assert lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(addr), *dims,
                                                 vkt.F32 if fmt is None else fmt, 1, 1, 1, 0, 1) == 0
        return h

    x, gy, gx = view(0x100000), view(0x200000), view(0x300000)
    other_dims, u8 = view(0x400000, (8, 8, 9)), view(0x500000, fmt=vkt.U8)
    f = vkt.Filter.gaussian(3, 1.0)
    gw = ctypes.c_void_p(0x600000)
    B = lib.vktApplyFilterBackwardSV
    assert B(gx, gw, None, x, f.handle) == 2
    assert B(gx, gw, gy, x, None) == 2
    assert B(gx, gw, gy, u8, f.handle) == 4               # float32 volumes only
    assert B(gx, gw, other_dims, x, f.handle) == 3
    assert B(other_dims, gw, gy, x, f.handle) == 3
    assert B(x, gw, gy, x, f.handle) == 1                 # dL/dx written over the source
    assert B(gy, gw, gy, x, f.handle) == 1                # ... or over dL/dy
    assert B(gx, ctypes.c_void_p(0x600002), gy, x, f.handle) == 1   # misaligned dL/dw
    assert B(gx, gw, gy, x, f.handle) == 6                # valid: reaches the device check
    assert B(None, gw, gy, x, f.handle) == 6
    N = lib.vktApplyFilterWeightGradNoAllocSV
    assert N(gw, None, x, f.handle) == 2
    assert N(None, gy, x, f.handle) == 1
    assert N(ctypes.c_void_p(0x600002), gy, x, f.handle) == 1
    assert N(gw, gy, u8, f.handle) == 4
    assert N(gw, other_dims, x, f.handle) == 3
    assert N(gw, gy, x, f.handle) == 6
    for h in (x, gy, gx, other_dims, u8):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_apply_filter_range_validation_without_device(vkt, lib):
    fake1, fake2 = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000)
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(a), fake1, 8, 6, 4, vkt.F32, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(b), fake2, 8, 6, 4, vkt.F32, 1, 1, 1, 0, 1) == 0
    f = vkt.Filter.gaussian(3, 1.0)
    R = lib.vktApplyFilterRangeSV
    assert R(None, a, f.handle, 0, 0, 0, 1, 1, 1) == 2
    for box in ((-1, 0, 0, 8, 6, 4), (0, 0, 0, 9, 6, 4), (0, 0, 0, 8, 7, 4), (0, 0, 0, 8, 6, 5),
                (3, 0, 0, 2, 6, 4), (0, 5, 0, 8, 4, 4), (0, 0, 3, 8, 6, 2)):
        assert R(a, b, f.handle, *box) == 1, box      # box outside the volume or reversed
    # a valid box reaches the device check (no GPU here)
    assert R(a, b, f.handle, 1, 1, 1, 7, 5, 3) == 6
    assert R(a, b, f.handle, 2, 0, 0, 2, 6, 4) == 6     # empty box: still needs a device
    for h in (a, b):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_brick_decompose_validation_without_device(vkt, lib):
    src = ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(src), ctypes.c_void_p(0x100000), 10, 7, 5,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    cx, cy, cz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    C = lib.vktBrickDecomposeCountSV
    assert C(ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(cz), src, 4, 7, 2) == 0
    assert (cx.value, cy.value, cz.value) == (3, 1, 3)
    assert C(ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(cz), src, 0, 7, 2) == 1
    assert C(ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(cz), None, 4, 7, 2) == 2
    # one brick of the whole volume with ghost 1: dims 12 x 9 x 7
    good, wrong_dims, wrong_fmt = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(good), ctypes.c_void_p(0x200000), 12, 9, 7,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(wrong_dims), ctypes.c_void_p(0x300000), 12, 9, 8,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(wrong_fmt), ctypes.c_void_p(0x400000), 12, 9, 7,
                                             vkt.F32, 1, 1, 1, 0, 1) == 0
    D = lib.vktBrickDecomposeSV
    arr = lambda *h: (ctypes.c_void_p * len(h))(*(x.value for x in h))
    assert D(arr(good), 1, src, 10, 7, 5, -1) == 1          # negative ghost
    assert D(arr(good), 2, src, 10, 7, 5, 1) == 1           # count mismatch
    assert D(arr(wrong_dims), 1, src, 10, 7, 5, 1) == 3     # brick dims
    assert D(arr(wrong_fmt), 1, src, 10, 7, 5, 1) == 1      # brick format
    assert D(arr(src), 1, src, 10, 7, 5, 0) == 1            # the source itself (overlap)
    assert D(arr(good), 1, src, 10, 7, 5, 1) == 6           # valid: reaches the device check
    for h in (src, good, wrong_dims, wrong_fmt):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_batch_validation_without_device(vkt, lib):
    """The triples of a batch run at once: no destination may overlap another destination
    or any source of the batch, while sources may be shared."""
    nbytes = 8 * 8 * 8 * 4

    def view(addr):
        h = ctypes.c_void_p()
        assert lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(addr), 8, 8, 8,
                                                 vkt.F32, 1, 1, 1, 0, 1) == 0
        return h

    a, b, c, d = (view(x) for x in (0x100000, 0x200000, 0x300000, 0x400000))
    touching = view(0x100000 + nbytes)         # starts where a ends: no overlap
    straddling = view(0x100000 + nbytes - 4)   # shares a's last voxel
    f = vkt.Filter.gaussian(3, 1.0)
    arr = lambda *h: (ctypes.c_void_p * len(h))(*(x.value for x in h))
    B = lambda dst, src: lib.vktApplyFilterBatchSV(len(dst), arr(*dst), arr(*src),
                                                   arr(*([f.handle] * len(dst))))
    assert lib.vktApplyFilterBatchSV(0, arr(a), arr(b), arr(f.handle)) == 1
    assert B([a, c], [b, ctypes.c_void_p()]) == 2   # NULL source handle
    assert B([a, c], [b, d]) == 6              # valid: reaches the device check
    assert B([a, c], [b, b]) == 6              # a shared source is fine
    assert B([a, a], [b, d]) == 1              # one destination written twice
    assert B([a, c], [b, a]) == 1              # a destination read by another triple
    assert B([c, a], [a, d]) == 1              # the same, other order
    assert B([a, touching], [b, d]) == 6
    assert B([a, straddling], [b, d]) == 1     # destinations overlap by one voxel
    assert B([c, d], [straddling, b]) == 6     # sources may overlap each other
    assert B([c, b], [d, straddling]) == 6
    assert B([straddling, c], [b, a]) == 1     # a destination overlaps another triple's source
    for h in (a, b, c, d, touching, straddling):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_clahe_validation_without_device(vkt, lib):
    a, b, f = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(a), ctypes.c_void_p(0x100000), 16, 8, 4,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(b), ctypes.c_void_p(0x200000), 16, 8, 4,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(f), ctypes.c_void_p(0x300000), 16, 8, 4,
                                             vkt.F32, 1, 1, 1, 0, 1) == 0
    C = lib.vktClahe3DSV
    assert C(None, a, 2, 2, 2, 2.0) == 2
    assert C(f, a, 2, 2, 2, 2.0) == 4            # not uint8
    assert C(b, a, 3, 2, 2, 2.0) == 1            # 3 does not divide 16
    assert C(b, a, 2, 0, 2, 2.0) == 1
    assert C(a, a, 2, 2, 2, 2.0) == 1            # overlapping
    assert C(b, a, 4, 4, 2, 2.0) == 6            # valid: reaches the device check
    for h in (a, b, f):
        assert lib.vktStructuredVolumeDestroy(h) == 0


@without_device
def test_render_validation_without_device(vkt, lib):
    import numpy as np
    v = ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(v), ctypes.c_void_p(0x100000), 8, 8, 8,
                                             vkt.U8, 1, 1, 1, 0, 1) == 0
    lut = np.array([[0, 0, 0, 0], [1, 1, 1, 1]], dtype=np.float32)

    def params(**kw):
        p = vkt.RenderParams()
        p.eye[:] = kw.get("eye", (4, 4, -10))
        p.center[:] = (4, 4, 4)
        p.up[:] = kw.get("up", (0, 1, 0))
        p.fovy, p.step, p.termination = kw.get("fovy", 0.8), kw.get("step", 0.5), 2.0
        p.background[:] = (0, 0, 0, 0)
        p.lutSize = kw.get("n", 2)
        p.lut = lut.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        return ctypes.cast(ctypes.pointer(p), ctypes.c_void_p), p

    img = ctypes.c_void_p(0x400000)
    R = lib.vktRenderSV
    for kw in (dict(up=(0, 0, 1)), dict(step=0.0), dict(fovy=0.0), dict(fovy=3.5), dict(n=1),
               dict(n=257), dict(eye=(4, 4, 4))):
        ptr, keep = params(**kw)
        assert R(img, 8, 8, v, ptr) == 1, kw
    ptr, keep = params()
    assert R(img, 0, 8, v, ptr) == 1
    assert R(ctypes.c_void_p(0x400004), 8, 8, v, ptr) == 1     # image not 16-byte aligned
    assert R(img, 8, 8, None, ptr) == 2
    assert R(img, 8, 8, v, ptr) == 6                            # valid: reaches the device check
    assert lib.vktStructuredVolumeDestroy(v) == 0


@pytest.mark.gpu
def test_view_refuses_host_memory(vkt, lib):
    """CreateView checks the pointer it is given: host memory (pageable or pinned) is
    refused with INVALID_VALUE, device memory of the current device is accepted; the check
    launches nothing."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    before = vkt.launch_count()
    host = ctypes.create_string_buffer(4096 + 16)        # pageable host memory
    addr = (ctypes.addressof(host) + 15) // 16 * 16
    h = ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(addr), 16, 16, 16,
                                             vkt.U8, 1, 1, 1, 0, 1) == 1
    assert not h.value
    pinned = torch.empty(4096, dtype=torch.uint8).pin_memory()
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(pinned.data_ptr()),
                                             16, 16, 16, vkt.U8, 1, 1, 1, 0, 1) == 1
    dev = torch.empty(4096, dtype=torch.uint8, device="cuda")
    assert lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(dev.data_ptr()),
                                             16, 16, 16, vkt.U8, 1, 1, 1, 0, 1) == 0
    assert lib.vktStructuredVolumeDestroy(h) == 0
    assert vkt.launch_count() == before


def test_owning_create_reports_missing_device(vkt, lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert lib.vktStructuredVolumeCreate(ctypes.byref(h), 4, 4, 4, vkt.F32, 1, 1, 1, 0, 1) == 6


def test_filter_validation(vkt, lib):
    h = ctypes.c_void_p()
    for k in (0, 2, 4, 11, -1):
        assert lib.vktFilterCreate(ctypes.byref(h), k, None) == 4
    assert lib.vktFilterCreateGaussian(ctypes.byref(h), 3, 0.0) == 1
    assert lib.vktFilterCreateGaussian(ctypes.byref(h), 3, -1.0) == 1
    f = vkt.Filter.dense(np.zeros((3, 3, 3)))
    assert not f.is_separable
    with pytest.raises(vkt.VktError):
        f.normalize()                      # zero sum
    with pytest.raises(vkt.VktError):
        f.separable_weights()
    assert lib.vktFilterDestroy(None) == 2


@pytest.mark.parametrize("k,sigma", [(3, 1.0), (5, 1.5), (7, 7 / 3), (9, 3.0)])
def test_gaussian_filter_matches_oracle_construction(vkt, k, sigma):
    sigma = float(np.float32(sigma))      # the C ABI takes sigma as a float
    f = vkt.Filter.gaussian(k, sigma)
    assert f.k == k and f.is_separable
    gx, gy, gz = f.separable_weights()
    g = oracle.gaussian_1d(k, sigma)
    assert np.array_equal(gx, g) and np.array_equal(gy, g) and np.array_equal(gz, g)
    dense = f.weights()
    assert np.allclose(dense, oracle.gaussian_weights(k, sigma), rtol=1e-6, atol=0)


def test_dense_roundtrip_and_normalize(vkt):
    w = np.arange(27, dtype=np.float32).reshape(3, 3, 3) + 1
    f = vkt.Filter.dense(w)
    assert np.array_equal(f.weights(), w)
    f.normalize()
    assert math.isclose(float(f.weights().astype(np.float64).sum()), 1.0, rel_tol=1e-6)
    np.testing.assert_allclose(f.weights(), (w / w.astype(np.float64).sum()).astype(np.float32))
    f.set_weights(w * 2)
    assert np.array_equal(f.weights(), w * 2)


def test_separable_normalize_each_vector(vkt):
    f = vkt.Filter.separable([1, 2, 1], [1, 1, 1], [0, 4, 0])
    f.normalize()
    gx, gy, gz = f.separable_weights()
    assert np.allclose(gx, [0.25, 0.5, 0.25]) and np.allclose(gy, 1 / 3) and np.allclose(gz, [0, 1, 0])
    assert np.allclose(f.weights().sum(), 1.0)
