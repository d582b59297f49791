"""GPU parity of the backward pass against the FP64 oracle.

dL/dx is the exact adjoint of the clamp-to-edge correlation (taps beyond a face fold onto
the face voxel); dL/dw[d] = sum_i gy(i) x(clamp(i+d)).  Tolerances: gx within
1e-5 * sum|w| * max|gy|; gw within 1e-5 * sum|gy| * max|x| (the bound on any entry)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 5
TOL = 1e-5


def gpu_backward(x, gy, w, need_x=True, need_w=True):
    xt = torch.from_numpy(x).cuda()
    gyt = torch.from_numpy(gy.astype(np.float32)).cuda()
    gx = torch.empty_like(xt) if need_x else None
    gw = torch.empty(w.size, dtype=torch.float32, device="cuda") if need_w else None
    f = vkt.Filter.dense(w.astype(np.float32))
    vkt.apply_filter_backward(vkt.StructuredVolume.from_tensor(gx) if need_x else None, gw,
                              vkt.StructuredVolume.from_tensor(gyt),
                              vkt.StructuredVolume.from_tensor(xt), f)
    torch.cuda.synchronize()
    vkt.synchronize()
    return (gx.cpu().numpy() if need_x else None), (gw.cpu().numpy().reshape(w.shape) if need_w else None)


SHAPES = [(21, 40, 72), (13, 37, 70), (3, 5, 4), (1, 1, 9), (40, 2, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_backward_matches_oracle(shape, k):
    x = synth.uniform(SEED + k, shape, -1.0, 1.0)
    gy = synth.uniform(SEED + 10 + k, shape, -1.0, 1.0).astype(np.float64)
    w = synth.normal(SEED + 20 + k, (k, k, k), 0.0, 1.0).astype(np.float64)
    w32 = w.astype(np.float32)
    gx, gw = gpu_backward(x, gy.astype(np.float32), w32)
    rx, rw = oracle.correlate_backward(x, gy.astype(np.float32).astype(np.float64), w32)
    sx = np.abs(w32.astype(np.float64)).sum() * np.abs(gy).max()
    ex = np.max(np.abs(gx - rx)) / sx
    assert ex <= TOL, f"gx error {ex:.2e}"
    sw = np.abs(gy).sum() * np.abs(x).max()
    ew = np.max(np.abs(gw - rw)) / sw
    assert ew <= TOL, f"gw error {ew:.2e}"


def test_adjoint_identity_on_gpu():
    shape = (30, 50, 64)
    x = synth.uniform(SEED + 30, shape, -1.0, 1.0)
    y = synth.uniform(SEED + 31, shape, -1.0, 1.0)
    w = synth.normal(SEED + 32, (5, 5, 5)).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    cx = vkt.filter_tensor(xt, vkt.Filter.dense(w), path="direct")
    gx, _ = gpu_backward(x, y, w, need_w=False)
    lhs = float(torch.sum(cx.double() * yt.double()))
    rhs = float(np.sum(x.astype(np.float64) * gx))
    assert abs(lhs - rhs) <= 1e-5 * np.abs(w).sum() * x.size


def test_gradient_only_weights_or_only_input():
    shape = (9, 20, 24)
    x = synth.uniform(SEED + 40, shape)
    gy = synth.uniform(SEED + 41, shape)
    w = synth.normal(SEED + 42, (3, 3, 3)).astype(np.float32)
    _, gw = gpu_backward(x, gy, w, need_x=False)
    gx, _ = gpu_backward(x, gy, w, need_w=False)
    rx, rw = oracle.correlate_backward(x, gy.astype(np.float64), w)
    assert np.max(np.abs(gw - rw)) <= TOL * np.abs(gy).sum()
    assert np.max(np.abs(gx - rx)) <= TOL * np.abs(w).sum()


def test_training_config_autograd():
    """8 x 128^3 float32 blob volumes, learnable 5^3 kernel N(0,0.1), target filtered by a
    hidden 5^3 kernel N(0,0.1), MSE loss; forward + backward through autograd."""
    B, n, k = 8, 128, 5
    vols = np.stack([synth.blobs(SEED + 100 + b, (n, n, n)) for b in range(B)])
    w0 = synth.normal(SEED + 200, (k, k, k), 0.0, 0.1)
    wh = synth.normal(SEED + 201, (k, k, k), 0.0, 0.1)
    xt = torch.from_numpy(vols).cuda().requires_grad_(True)
    wt = torch.from_numpy(w0).cuda().requires_grad_(True)
    with torch.no_grad():
        target = vkt.apply_filter_autograd(xt.detach(), torch.from_numpy(wh).cuda(), "direct")
    y = vkt.apply_filter_autograd(xt, wt, "direct")
    loss = torch.mean((y - target) ** 2)
    loss.backward()
    torch.cuda.synchronize()
    gw = wt.grad.cpu().numpy()
    gx = xt.grad.cpu().numpy()
    # oracle gradient on volumes 0 and 7 (gw summed over the batch: check the sum)
    rw_total = np.zeros((k, k, k))
    gy_all = (2.0 / (B * n ** 3)) * (y.detach().double() - target.double()).cpu().numpy()
    idx = np.random.default_rng(1).integers(0, n ** 3, 20000)
    for b in range(B):
        _, rw = oracle.correlate_backward(vols[b], gy_all[b], w0, need_gx=False)
        rw_total += rw
        if b in (0, B - 1):
            rx = oracle.backward_input_points(gy_all[b], w0, idx)
            sx = np.abs(w0.astype(np.float64)).sum() * np.abs(gy_all[b]).max()
            assert np.max(np.abs(gx[b].ravel()[idx] - rx)) / sx <= TOL
    sw = sum(np.abs(gy_all[b]).sum() * np.abs(vols[b]).max() for b in range(B))
    assert np.max(np.abs(gw - rw_total)) / sw <= TOL
    # central differences of the GPU loss in w (float32 forward, h = 1e-3): loose check
    h = 1e-3
    for d in (0, 62, 124):
        e = np.zeros(k ** 3, np.float32)
        e[d] = h
        with torch.no_grad():
            lp = torch.mean((vkt.apply_filter_autograd(xt.detach(), wt.detach() + torch.from_numpy(e.reshape(w0.shape)).cuda(), "direct") - target).double() ** 2)
            lm = torch.mean((vkt.apply_filter_autograd(xt.detach(), wt.detach() - torch.from_numpy(e.reshape(w0.shape)).cuda(), "direct") - target).double() ** 2)
        fd = float(lp - lm) / (2 * h)
        assert abs(fd - gw.ravel()[d]) <= 2e-3 * max(abs(gw.ravel()[d]), np.abs(gw).max()), (d, fd, gw.ravel()[d])
