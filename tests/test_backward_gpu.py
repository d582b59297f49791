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


# the last two are thinner than the k = 9 filter's 4-voxel halo on two axes, so the adjoint's
# shell folds several layers onto the same face voxels
SHAPES = [(21, 40, 72), (13, 37, 70), (3, 5, 4), (1, 1, 9), (40, 2, 3), (2, 3, 2), (9, 1, 17)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 3, 5, 7, 9])
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


def _views_in(buf, offsets, shape):
    """Volume views of `shape` at the given element offsets of one flat CUDA buffer."""
    n = int(np.prod(shape))
    ts = [buf[o:o + n].view(shape) for o in offsets]
    return ts, [vkt.StructuredVolume.from_tensor(t) for t in ts]


@pytest.mark.parametrize("shape", [(21, 34, 72), (13, 30, 70)])
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("layout", ["even", "uneven"])
def test_backward_batch_matches_oracle(shape, k, layout):
    """vktApplyFilterBackwardBatchSV over 3 volumes: dL/dx per volume and dL/dw summed over
    the batch, against the oracle.  'even': the volumes of one batch tensor (one launch per
    kernel); 'uneven': volumes at irregular offsets (one launch per volume, one reduction)."""
    B = 3
    vox = int(np.prod(shape))
    offs = [b * vox for b in range(B)] if layout == "even" else [0, vox + 64, 2 * vox + 192]
    size = offs[-1] + vox
    xs = [synth.uniform(SEED + 300 + b, shape, -1.0, 1.0) for b in range(B)]
    gys = [synth.uniform(SEED + 310 + b, shape, -1.0, 1.0) for b in range(B)]
    w = synth.normal(SEED + 320 + k, (k, k, k)).astype(np.float32)
    xbuf = torch.zeros(size, dtype=torch.float32, device="cuda")
    gybuf = torch.zeros(size, dtype=torch.float32, device="cuda")
    gxbuf = torch.full((size,), 7.0, dtype=torch.float32, device="cuda")
    xt, vx = _views_in(xbuf, offs, shape)
    gyt, vgy = _views_in(gybuf, offs, shape)
    gxt, vgx = _views_in(gxbuf, offs, shape)
    for b in range(B):
        xt[b].copy_(torch.from_numpy(xs[b]))
        gyt[b].copy_(torch.from_numpy(gys[b]))
    gw = torch.full((k ** 3,), float("nan"), dtype=torch.float32, device="cuda")
    f = vkt.Filter.dense(w)
    vkt.apply_filter_backward_batch(vgx, gw, vgy, vx, f)
    torch.cuda.synchronize()
    vkt.synchronize()
    rw_total = np.zeros((k, k, k))
    for b in range(B):
        rx, rw = oracle.correlate_backward(xs[b], gys[b].astype(np.float64), w)
        rw_total += rw
        err = np.max(np.abs(gxt[b].cpu().numpy() - rx)) / (np.abs(w).sum() * np.abs(gys[b]).max())
        assert err <= TOL, (b, err)
    sw = sum(np.abs(gys[b]).sum() * np.abs(xs[b]).max() for b in range(B))
    assert np.max(np.abs(gw.cpu().numpy().reshape(w.shape) - rw_total)) / sw <= TOL
    if layout == "uneven":      # the gaps between the volumes are untouched
        g = gxbuf.cpu().numpy()
        assert np.all(g[vox:vox + 64] == 7.0) and np.all(g[2 * vox + 64:2 * vox + 192] == 7.0)


def test_backward_batch_weights_only_and_rejections():
    shape, B, k = (9, 16, 32), 2, 3
    x = torch.from_numpy(np.stack([synth.uniform(SEED + 330 + b, shape, -1.0, 1.0) for b in range(B)])).cuda()
    gy = torch.from_numpy(np.stack([synth.uniform(SEED + 340 + b, shape, -1.0, 1.0) for b in range(B)])).cuda()
    w = synth.normal(SEED + 350, (k, k, k)).astype(np.float32)
    f = vkt.Filter.dense(w)
    vx = [vkt.StructuredVolume.from_tensor(x[b]) for b in range(B)]
    vgy = [vkt.StructuredVolume.from_tensor(gy[b]) for b in range(B)]
    gw = torch.empty(k ** 3, dtype=torch.float32, device="cuda")
    vkt.apply_filter_backward_batch(None, gw, vgy, vx, f)
    torch.cuda.synchronize()
    ref = sum(oracle.correlate_backward(x[b].cpu().numpy(), gy[b].double().cpu().numpy(), w,
                                        need_gx=False)[1] for b in range(B))
    sw = float(gy.abs().sum()) * float(x.abs().max())
    assert np.max(np.abs(gw.cpu().numpy().reshape(w.shape) - ref)) / sw <= TOL
    # a gradient volume that overlaps a source is refused
    with pytest.raises(vkt.VktError) as e:
        vkt.apply_filter_backward_batch([vx[1], vkt.StructuredVolume.from_tensor(torch.empty_like(x[0]))],
                                        None, vgy, vx, f)
    assert e.value.code == 1
    # dims must agree across the batch
    other = torch.zeros((9, 16, 36), device="cuda")
    with pytest.raises(vkt.VktError) as e:
        vkt.apply_filter_backward_batch(None, gw, [vgy[0], vkt.StructuredVolume.from_tensor(other)], vx, f)
    assert e.value.code == 3


@pytest.mark.parametrize("dfmt", ["f32", "u16"])
@pytest.mark.parametrize("layout", ["even", "uneven"])
def test_forward_batch_one_filter(dfmt, layout):
    """vktApplyFilterBatchSV with one dense filter over 4 equal uint8 volumes: a single
    direct launch when the volumes are evenly spaced; uint16 codes bit-exact outside the tie
    window (compensated accumulation)."""
    from gpu_util import compare
    B, shape, k = 4, (23, 40, 72), 3
    vox = int(np.prod(shape))
    srcs = [synth.quantize(synth.uniform(SEED + 360 + b, shape), synth.U8) for b in range(B)]
    w = synth.normal(SEED + 370, (k, k, k)).astype(np.float32)
    offs = [b * vox for b in range(B)] if layout == "even" else [0, vox + 32, 2 * vox + 48, 3 * vox + 96]
    size = offs[-1] + vox
    sbuf = torch.zeros(size * 4, dtype=torch.uint8, device="cuda")     # room for any layout
    st, vs = _views_in(sbuf, offs, shape)
    for b in range(B):
        st[b].copy_(torch.from_numpy(srcs[b]))
    dt = torch.float32 if dfmt == "f32" else torch.uint16
    dbuf = torch.empty(size, dtype=dt, device="cuda")
    n = int(np.prod(shape))
    dts = [dbuf[o:o + n].view(shape) for o in offs]
    drange = (0.0, 1.0) if dfmt == "f32" else (-4.0, 9.0)
    vd = [vkt.StructuredVolume.from_tensor(t, *drange) for t in dts]
    f = vkt.Filter.dense(w)
    before = vkt.launch_count()
    vkt.apply_filter_batch(vd, vs, [f] * B)
    launched = vkt.launch_count() - before
    torch.cuda.synchronize()
    vkt.synchronize()
    if layout == "even":
        assert launched == 1
    for b in range(B):
        ref = oracle.correlate(srcs[b], w.astype(np.float64), 0.0, 1.0)
        compare(dts[b].cpu().numpy(), ref, w, srcs[b], (0.0, 1.0), drange, f"batch volume {b}")


def test_short_z_chunks_direct_adjoint_weight_gradient(capfd):
    """A volume too small for one CTA per SM runs z chunks shorter than the filter's 2r halo
    (down to one plane) in the forward, adjoint and weight-gradient kernels: all three
    against the oracle, and the chunk lengths read from the debug log."""
    shape, k = (40, 30, 60), 9
    x = synth.uniform(SEED + 380, shape, -1.0, 1.0)
    gy = synth.uniform(SEED + 381, shape, -1.0, 1.0).astype(np.float64)
    w = synth.normal(SEED + 382, (k, k, k)).astype(np.float32)
    f = vkt.Filter.dense(w)
    xt = torch.from_numpy(x).cuda()
    with vkt.policy(path="direct", debug=vkt.DEBUG_LOG):
        y = vkt.filter_tensor(xt, f)
        gx, gw = gpu_backward(x, gy, w)
    torch.cuda.synchronize()
    log = capfd.readouterr().err
    import re
    chunks = {m.group(1): int(m.group(2)) for m in
              re.finditer(r"\[vkt\] (direct|direct-adjoint|wgrad) k=9 .*?zchunk=(\d+)", log)}
    assert set(chunks) == {"direct", "direct-adjoint", "wgrad"}, log
    assert all(z < k - 1 for z in chunks.values()), chunks
    ref = oracle.correlate(x, w.astype(np.float64))
    assert np.max(np.abs(y.cpu().numpy() - ref)) / (np.abs(w).sum() * np.abs(x).max()) <= TOL
    rx, rw = oracle.correlate_backward(x, gy, w)
    assert np.max(np.abs(gx - rx)) / (np.abs(w).sum() * np.abs(gy).max()) <= TOL
    assert np.max(np.abs(gw - rw)) / (np.abs(gy).sum() * np.abs(x).max()) <= TOL
