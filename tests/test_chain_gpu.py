"""GPU: calls enqueued back to back on one stream, each reading what the previous one wrote.

The direct and separable kernels are launched with programmatic stream serialization, so
a call's CTAs may start while the previous call is still running; they must not read their
source (written by that call) or overwrite their destination (read by it) before the
previous grid is complete.  A chain of filters over two ping-pong buffers, with no host
synchronisation between the calls, checks both orders against the FP64 oracle applied in
the same sequence.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 41


def _gaussian_dense(k, sigma):
    g = oracle.gaussian_1d(k, sigma)
    return np.einsum("i,j,l->ijl", g, g, g)


@pytest.mark.parametrize("shape", [(40, 70, 144), (23, 45, 150), (64, 64, 64)])
def test_chain_of_calls_reads_each_previous_output(shape):
    x0 = synth.uniform(SEED + shape[0], shape, 0.0, 1.0).astype(np.float32)
    lap = synth.laplacian_3()
    # (filter, path, dense weights for the oracle): normalised Gaussians keep the values in
    # range; the Laplacian (scaled by 1/8) exercises signed weights between them
    steps = [
        (vkt.Filter.gaussian(3, 1.0), "direct", None),
        (vkt.Filter.gaussian(5, 1.5), "separable", None),
        (vkt.Filter.dense((lap / 8.0).astype(np.float32)), "direct", (lap / 8.0).astype(np.float32)),
        (vkt.Filter.gaussian(5, 1.2), "direct", None),
        (vkt.Filter.gaussian(3, 0.8), "separable", None),
        (vkt.Filter.gaussian(7, 2.0), "direct", None),
    ]
    bufs = [torch.from_numpy(x0).cuda(), torch.empty(shape, dtype=torch.float32, device="cuda")]
    vols = [vkt.StructuredVolume.from_tensor(b, 0.0, 1.0) for b in bufs]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    for i, (f, path, _) in enumerate(steps):
        vkt.apply_filter(vols[(i + 1) % 2], vols[i % 2], f, path=path, stream=stream)
    torch.cuda.synchronize()
    vkt.synchronize()
    gpu = bufs[len(steps) % 2].cpu().numpy().astype(np.float64)

    # the oracle takes each step's float32 input, as the GPU does (its buffers are float32)
    ref = x0
    for f, _, dense in steps:
        w = dense if dense is not None else f.weights()
        ref = oracle.correlate(ref.astype(np.float32), np.asarray(w, dtype=np.float64))
    err = np.max(np.abs(gpu - ref))
    # each step's FP32 error is within 1e-5 of sum|w| * max|input| (sum|w| <= 1 here)
    assert err <= 1e-5 * len(steps) * max(1.0, np.abs(ref).max()), f"chain error {err:.3e}"
