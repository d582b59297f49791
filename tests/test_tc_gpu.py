"""GPU parity of the tensor-core path (FP16 hi/lo split on tcgen05, FP32 accumulation)
against the FP64 oracle, at the same tolerance as the FP32 path: max |gpu - oracle| <=
1e-5 * sum|w| * max|x|.  Cases span several 16 x 128 tiles and z chunks, with ragged tails
on every axis, plus the 1024 x 1024 x 512 turbulence-like workload at full size (sampled)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FLOAT_TOL, compare, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 3


def kernel(k, seed, normalise=True):
    w, _ = synth.random_kernel(seed, k, 1.0, normalise_sum=normalise)
    return w


@pytest.mark.parametrize("k", [5, 7, 9])
@pytest.mark.parametrize("shape", [(40, 300, 100), (9, 130, 36), (3, 17, 4)])
def test_tensor_path_random_kernels(k, shape):
    src = synth.uniform(SEED + k, shape, -1.0, 1.0)
    w = kernel(k, SEED + 10 + k)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="tensor")
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), f"tensor k={k} {shape}")


@pytest.mark.parametrize("k", [7])
def test_tensor_path_wide_dynamic_range(k):
    """Values spanning many binades in one plane: the per-plane power-of-two scale and the
    lo half keep the error relative to max|x|."""
    shape = (20, 140, 48)
    src = synth.uniform(SEED + 40, shape, -1.0, 1.0)
    src *= np.float32(1e3) ** synth.uniform(SEED + 41, shape, -1.0, 1.0)
    w = kernel(k, SEED + 42)
    gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="tensor")
    ref = oracle.correlate(src, w)
    compare(gpu, ref, w, src, (0, 1), (0, 1), "tensor wide range")


def test_tensor_path_matches_direct_path_closely():
    shape = (33, 260, 80)
    src = synth.fourier(SEED + 50, (80, 260, 33))
    w = kernel(7, SEED + 51)
    a = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="tensor")
    b = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32, path="direct")
    scale = oracle.error_scale(w, float(np.abs(src).max()))
    assert np.max(np.abs(a.astype(np.float64) - b)) / scale < 2 * FLOAT_TOL


def test_tensor_path_rejects_unsupported():
    src = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    f = vkt.Filter.dense(np.ones((7, 7, 7), np.float32))
    with pytest.raises(vkt.VktError):
        vkt.filter_tensor(src, f, path="tensor", out=out)
    f3 = vkt.Filter.dense(np.ones((3, 3, 3), np.float32))
    with pytest.raises(vkt.VktError):
        vkt.filter_tensor(out.clone(), f3, path="tensor", out=out)


def _sample(shape, n, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, nz * ny * nx, n)]
    for axis, extent in enumerate(shape):
        for plane in (0, 1, 2, 3, extent - 4, extent - 3, extent - 2, extent - 1):
            c = [rng.integers(0, e, n // 32) for e in shape]
            c[axis] = np.full(n // 32, plane)
            idx.append((c[0] * ny + c[1]) * nx + c[2])
    return np.unique(np.concatenate(idx))


@pytest.fixture(scope="module")
def dns_field():
    return synth.volume("fourier", synth.F32, (1024, 1024, 512), SEED + 60)


@pytest.mark.parametrize("k,path", [(7, "tensor"), (9, "tensor"), (7, "direct")])
def test_full_size_turbulence_sampled(dns_field, k, path):
    """1024 x 1024 x 512 float32 field, normalised N(0,1) k^3 kernel, benchmark launch shape."""
    w = kernel(k, SEED + 70 + k)
    gpu = run_gpu(vkt, dns_field, vkt.Filter.dense(w), torch.float32, path=path)
    idx = _sample(dns_field.shape, 100000, SEED + 80)
    ref = oracle.correlate_points(dns_field, w, idx)
    err = compare(gpu.ravel()[idx], ref, w, dns_field, (0, 1), (0, 1), f"1024x1024x512 {path} k={k}")
    print(f"normalised max error {path} k={k}: {err:.3e}")
