"""GPU parity: the CUDA paths of ApplyFilter (through the C ABI) against the FP64 oracle.

Small cases span several bricks (64 x 32 outputs per CTA in x, y; z chunks) and a ragged
tail on every axis; full-size cases of the benchmark compare sampled voxels (all eight
corners, random face voxels and random interior voxels) with the oracle's per-voxel
evaluation.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED
DT = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}


def src_volume(fmt, shape, seed):
    nz, ny, nx = shape
    if fmt == synth.F32:
        return synth.uniform(seed, shape, -1.0, 2.0)
    return synth.quantize(synth.uniform(seed, shape), fmt)


def dense_filter(k, seed):
    w = synth.normal(seed, (k, k, k), 0.0, 1.0)
    return w


# shape (nz, ny, nx): first is TMA-describable for every format (nx multiple of 16), the
# second is not (rows not 16-byte multiples) and takes the plain-load path
SHAPES = [(37, 70, 144), (19, 45, 150)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 3, 5, 7, 9])
def test_direct_f32_random_kernel(shape, k):
    src = src_volume(synth.F32, shape, SEED + k)
    w = dense_filter(k, SEED + 100 + k)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="direct")
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), f"direct k={k} {shape}")


@pytest.mark.parametrize("sfmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("dfmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("k", [3, 5])
def test_direct_format_pairs(sfmt, dfmt, k):
    shape = SHAPES[0] if (sfmt + dfmt) % 2 == 0 else SHAPES[1]
    src = src_volume(sfmt, shape, SEED + 7 * sfmt + dfmt)
    g = oracle.gaussian_1d(k, 1.0)
    w = (oracle.separable_weights(g, g, g)).astype(np.float32)     # positive, sums to ~1
    srange, drange = (-0.5, 2.0), (-0.25, 1.75)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), DT[dfmt], srange, drange, path="direct")
    ref = oracle.correlate(src, w, *srange)
    compare(gpu, ref, w, src, srange, drange, f"direct {sfmt}->{dfmt} k={k}")


@pytest.mark.parametrize("sfmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("dfmt", [synth.U8, synth.U16])
def test_direct_laplacian_into_integer_codes(sfmt, dfmt):
    """The 7-point Laplacian (signed weights) into uint8 / uint16 codes with a shifted
    destination range: codes bit-exact outside the 1e-3 LSB tie window, negative results
    clamped to code 0."""
    shape = SHAPES[(sfmt + dfmt) % 2]
    src = src_volume(sfmt, shape, SEED + 110 + 3 * sfmt + dfmt)
    srange, drange = (0.0, 1.0), (-4.0, 9.0)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(synth.laplacian_3()), DT[dfmt], srange, drange,
                  path="direct")
    w = oracle.laplacian_3()
    ref = oracle.correlate(src, w, *srange)
    compare(gpu, ref, w, src, srange, drange, f"laplacian {sfmt}->{dfmt}")


@pytest.mark.parametrize("k", [3, 5, 7, 9])
@pytest.mark.parametrize("sfmt", [synth.U16, synth.F32])
def test_direct_uint16_destination_exact(k, sfmt):
    """Dense random kernels (N(0.3, 1), not normalised) into uint16 codes with shifted
    ranges: bit-exact outside the tie window, through the compensated accumulation."""
    shape = SHAPES[k % 2]
    src = src_volume(sfmt, shape, SEED + 120 + k + sfmt)
    w = synth.normal(SEED + 130 + k, (k, k, k), 0.3, 1.0).astype(np.float32)
    srange, drange = (-1.0, 3.0), (-40.0, 90.0)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.uint16, srange, drange, path="direct")
    ref = oracle.correlate(src, w, *srange)
    compare(gpu, ref, w, src, srange, drange, f"dense u16 dst k={k} src {sfmt}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 3, 5, 7, 9])
def test_separable_f32(shape, k):
    src = src_volume(synth.F32, shape, SEED + 20 + k)
    gx = synth.normal(SEED + 30 + k, (k,), 0.0, 1.0)
    gy = synth.normal(SEED + 40 + k, (k,), 0.0, 1.0)
    gz = synth.normal(SEED + 50 + k, (k,), 0.0, 1.0)
    f = vkt.Filter.separable(gx, gy, gz)
    gpu = run_gpu(vkt, src, f, torch.float32, path="separable")
    w = oracle.separable_weights(gx, gy, gz)
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), f"separable k={k} {shape}")


@pytest.mark.parametrize("sfmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("dfmt", [synth.U8, synth.U16, synth.F32])
def test_separable_gaussian_format_pairs(sfmt, dfmt):
    k, sigma = 5, 1.5
    shape = SHAPES[0] if (sfmt + dfmt) % 2 == 0 else SHAPES[1]
    src = src_volume(sfmt, shape, SEED + 60 + sfmt * 3 + dfmt)
    srange, drange = (0.0, 1.0), (0.0, 1.0)
    gpu = run_gpu(vkt, src, vkt.Filter.gaussian(k, sigma), DT[dfmt], srange, drange)
    w = oracle.gaussian_weights(k, sigma)
    ref = oracle.correlate(src, w, *srange)
    compare(gpu, ref, w, src, srange, drange, f"gaussian {sfmt}->{dfmt}")


@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_separable_uint16_destination_exact(k):
    """uint16 codes bit-exact outside the 1e-3 LSB tie window (compensated accumulation),
    with signed weights and shifted ranges."""
    shape = SHAPES[k % 2]
    src = src_volume(synth.U16, shape, SEED + 90 + k)
    g = [synth.normal(SEED + 95 + k + i, (k,), 0.3, 1.0) for i in range(3)]
    f = vkt.Filter.separable(*g)
    srange, drange = (-1.0, 3.0), (-4.0, 9.0)
    gpu = run_gpu(vkt, src, f, torch.uint16, srange, drange, path="separable")
    w = oracle.separable_weights(*g)
    ref = oracle.correlate(src, w, *srange)
    compare(gpu, ref, w, src, srange, drange, f"u16 dst k={k}")


EDGE_SHAPES = [(1, 1, 1), (1, 7, 3), (2, 3, 4), (1, 1, 1000), (300, 3, 5), (3, 260, 2)]


@pytest.mark.parametrize("shape", EDGE_SHAPES)
@pytest.mark.parametrize("path,k", [("direct", 3), ("direct", 7), ("separable", 5),
                                    ("separable", 9)])
def test_degenerate_shapes(shape, path, k):
    """Volumes thinner than the kernel: every tap clamps onto the faces."""
    src = src_volume(synth.F32, shape, SEED + 70)
    if path == "direct":
        w = dense_filter(k, SEED + 71)
        f = vkt.Filter.dense(w)
    else:
        g = [synth.normal(SEED + 72 + i, (k,)) for i in range(3)]
        f = vkt.Filter.separable(*g)
        w = oracle.separable_weights(*g)
    gpu = run_gpu(vkt, src, f, torch.float32, path=path)
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), f"{path} k={k} {shape}")


def test_smallest_config_uniform64_gaussian3_fp32_path():
    """64^3 float32, voxels i.i.d. U[0,1) from the seed, normalised 3^3 Gaussian sigma 1.0
    given as dense weights, FP32 CUDA-core (direct) path, every voxel against the oracle."""
    src = synth.volume("uniform", synth.F32, (64, 64, 64), synth.BASE_SEED)
    w = oracle.gaussian_weights(3, 1.0).astype(np.float32)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="direct")
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), "64^3 uniform gaussian3")
    # the same filter through the separable path and the automatic choice
    g = vkt.Filter.gaussian(3, 1.0)
    for path in ("separable", "auto"):
        gpu = run_gpu(vkt, src, g, torch.float32, path=path)
        compare(gpu, ref, w, src, (0, 1), (0, 1), f"64^3 uniform gaussian3 {path}")


def test_identity_and_constant_exact():
    shape = (33, 40, 72)
    src = src_volume(synth.F32, shape, SEED + 80)
    w = np.zeros((3, 3, 3), np.float32)
    w[1, 1, 1] = 1.0
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="direct")
    assert np.array_equal(gpu, src)
    c = np.full(shape, 0.375, np.float32)
    gpu = run_gpu(vkt, c, vkt.Filter.gaussian(5, 1.5), torch.float32)
    assert np.max(np.abs(gpu - 0.375)) < 1e-6


def test_paper_fillrange_example_blurred():
    """The C99 listing's 64^3 uint8 volume, FillRange(1,1,1 .. 63,63,63) = 1.0, blurred."""
    vol = np.zeros((64, 64, 64), np.uint8)
    vol[1:63, 1:63, 1:63] = 255
    f = vkt.Filter.gaussian(3, 1.0)
    gpu = run_gpu(vkt, vol, f, torch.float32)
    ref = oracle.correlate(vol, oracle.gaussian_weights(3, 1.0), 0.0, 1.0)
    compare(gpu, ref, oracle.gaussian_weights(3, 1.0), vol, (0, 1), (0, 1), "fillrange")


def _sample_indices(shape, n, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, nz * ny * nx, n)]
    for axis, extent in enumerate(shape):           # voxels on and next to every face
        for plane in (0, 1, extent - 2, extent - 1):
            c = [rng.integers(0, e, n // 16) for e in shape]
            c[axis] = np.full(n // 16, max(0, min(extent - 1, plane)))
            idx.append((c[0] * ny + c[1]) * nx + c[2])
    corners = [((z * ny) + y) * nx + x for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    idx.append(np.array(corners))
    return np.unique(np.concatenate(idx))


@pytest.fixture(scope="module")
def ct512():
    v = synth.volume("blobs", synth.U8, (512, 512, 512), SEED + 1)
    return v


@pytest.mark.parametrize("which", ["gaussian5", "laplacian3"])
def test_full_size_ct_512_sampled(ct512, which):
    """The 512^3 uint8 CT-like workload, at full size, in the benchmark's launch shape."""
    if which == "gaussian5":
        f = vkt.Filter.gaussian(5, 1.5)
        w = oracle.gaussian_weights(5, 1.5)
    else:
        w = oracle.laplacian_3()
        f = vkt.Filter.dense(synth.laplacian_3())
    gpu = run_gpu(vkt, ct512, f, torch.float32)
    idx = _sample_indices(ct512.shape, 200000, SEED + 90)
    ref = oracle.correlate_points(ct512, w, idx, 0.0, 1.0)
    compare(gpu.ravel()[idx], ref, w, ct512, (0, 1), (0, 1), f"512^3 {which}")
