"""GPU parity of the range version of ApplyFilter (vktApplyFilterRangeSV): inside the box the
oracle's full-volume correlation (taps read the real neighbours, clamped at the volume's
faces), outside it the destination's previous contents, bit for bit.

Boxes start and end off every tile and alignment boundary (x tiles are 64 wide and start on
a 16-byte boundary left of the box), touch the faces, or shrink to a column or one voxel;
shapes take both the tensor-map path (rows a multiple of 16 bytes) and the row-copy path.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 700
DT = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}
NP = {synth.U8: np.uint8, synth.U16: np.uint16, synth.F32: np.float32}


def source(fmt, shape, seed):
    if fmt == synth.F32:
        return synth.uniform(seed, shape, -1.0, 2.0)
    return synth.quantize(synth.uniform(seed, shape), fmt)


def prior(fmt, shape, seed):
    """The destination's contents before the call (must survive outside the box)."""
    if fmt == synth.F32:
        return synth.uniform(seed, shape, 5.0, 9.0)
    return synth.quantize(synth.uniform(seed, shape), fmt)


def make_filter(kind, k, seed):
    if kind == "separable":
        sigma = float(np.float32(k / 3.0))
        return vkt.Filter.gaussian(k, sigma), oracle.gaussian_weights(k, sigma)
    w = synth.normal(seed, (k, k, k), 0.0, 1.0).astype(np.float32)
    return vkt.Filter.dense(w), w.astype(np.float64)


def run_range(src, dst_fmt, filt, box, init, path="auto"):
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    out = torch.from_numpy(np.ascontiguousarray(init)).cuda()
    first, last = box
    vkt.filter_tensor(s, filt, out=out, path=path, roi=(first, last))
    torch.cuda.synchronize()
    vkt.synchronize()
    return out.cpu().numpy()


def check(gpu, init, src, w, box, what):
    (x0, y0, z0), (x1, y1, z1) = box
    inside = np.zeros(gpu.shape, dtype=bool)
    inside[z0:z1, y0:y1, x0:x1] = True
    assert np.array_equal(gpu[~inside], init[~inside]), f"{what}: voxels outside the box changed"
    if inside.any():
        ref = oracle.correlate(src, w, 0.0, 1.0)[z0:z1, y0:y1, x0:x1]
        compare(np.ascontiguousarray(gpu[z0:z1, y0:y1, x0:x1]), ref, w,
                src, (0.0, 1.0), (0.0, 1.0), what)


# (nz, ny, nx): rows of 96 bytes (u8) / 384 (f32) take tensor maps; 75-wide rows take copies
SHAPES = [(23, 70, 96), (19, 41, 75)]
BOXES = [
    ((3, 5, 2), (70, 61, 20)),      # interior, every bound off a tile / alignment boundary
    ((0, 0, 0), (96, 70, 23)),      # the whole volume (clipped per shape below)
    ((17, 0, 4), (18, 70, 9)),      # a one-voxel-wide column through the y faces
    ((40, 33, 11), (41, 34, 12)),   # a single voxel
    ((63, 9, 0), (75, 40, 19)),     # crosses the first 64-wide tile boundary, touches +x face
]


def clip(box, shape):
    nz, ny, nx = shape
    (x0, y0, z0), (x1, y1, z1) = box
    x1, y1, z1 = min(x1, nx), min(y1, ny), min(z1, nz)
    return (min(x0, x1), min(y0, y1), min(z0, z1)), (x1, y1, z1)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind,k", [("dense", 3), ("dense", 5), ("separable", 3), ("separable", 5),
                                    ("separable", 7)])
@pytest.mark.parametrize("sfmt,dfmt", [(synth.U8, synth.F32), (synth.F32, synth.F32),
                                       (synth.U8, synth.U8), (synth.U16, synth.U16)])
def test_range_matches_oracle_inside_and_keeps_outside(shape, kind, k, sfmt, dfmt):
    src = source(sfmt, shape, SEED + k)
    filt, w = make_filter(kind, k, SEED + 31 * k)
    for j, b in enumerate(BOXES):
        box = clip(b, shape)
        init = prior(dfmt, shape, SEED + 100 + j)
        gpu = run_range(src, dfmt, filt, box, init)
        check(gpu, init, src, w, box, f"{kind} k={k} {sfmt}->{dfmt} {shape} box {box}")


@pytest.mark.parametrize("kind,k", [("dense", 3), ("separable", 5)])
def test_whole_volume_range_equals_apply_filter(kind, k):
    shape = (21, 50, 80)
    src = source(synth.U8, shape, SEED + 5)
    filt, _ = make_filter(kind, k, SEED + 9)
    s = torch.from_numpy(src).cuda()
    full = vkt.filter_tensor(s, filt)
    ranged = vkt.filter_tensor(s, filt, out=torch.zeros_like(full),
                               roi=((0, 0, 0), (shape[2], shape[1], shape[0])))
    torch.cuda.synchronize()
    assert torch.equal(full, ranged)


def test_empty_box_writes_nothing_and_tensor_path_is_refused():
    shape = (12, 20, 32)
    src = torch.from_numpy(source(synth.F32, shape, SEED + 2)).cuda()
    init = torch.from_numpy(prior(synth.F32, shape, SEED + 3)).cuda()
    out = init.clone()
    filt = vkt.Filter.dense(synth.normal(SEED + 4, (5, 5, 5)).astype(np.float32))
    vkt.filter_tensor(src, filt, out=out, roi=((4, 4, 4), (4, 10, 10)))
    torch.cuda.synchronize()
    assert torch.equal(out, init)
    with pytest.raises(vkt.VktError) as e:
        vkt.filter_tensor(src, filt, out=out, path="tensor", roi=((0, 0, 0), (8, 8, 8)))
    assert e.value.code == 4     # VKT_ERROR_UNSUPPORTED


def test_range_full_size_sampled():
    """The bench's region, 300 x 250 x 270 voxels off every boundary of the 512^3 uint8
    CT-like volume, both filters of the benchmark step: seeded voxels inside the box
    against the oracle's per-voxel evaluation, voxels outside unchanged."""
    src = synth.volume("blobs", synth.U8, (512, 512, 512), synth.BASE_SEED + 1)
    (x0, y0, z0), (x1, y1, z1) = (101, 77, 130), (401, 327, 400)
    s = torch.from_numpy(src).cuda()
    rng = np.random.default_rng(SEED + 77)
    n = 4000
    idx = np.stack([rng.integers(z0, z1, n), rng.integers(y0, y1, n), rng.integers(x0, x1, n)], axis=1)
    # the box's corners and faces
    corners = np.array([[z, y, x] for z in (z0, z1 - 1) for y in (y0, y1 - 1) for x in (x0, x1 - 1)])
    idx = np.concatenate([corners, idx])
    outside = np.stack([rng.integers(0, 512, n), rng.integers(0, 512, n), rng.integers(0, 512, n)], axis=1)
    keep = ~((outside[:, 0] >= z0) & (outside[:, 0] < z1) & (outside[:, 1] >= y0) & (outside[:, 1] < y1)
             & (outside[:, 2] >= x0) & (outside[:, 2] < x1))
    outside = outside[keep]
    for filt, w in ((vkt.Filter.gaussian(5, 1.5), oracle.gaussian_weights(5, float(np.float32(1.5)))),
                    (vkt.Filter.dense(synth.laplacian_3()), oracle.laplacian_3())):
        out = torch.full(src.shape, -3.0, dtype=torch.float32, device="cuda")
        vkt.filter_tensor(s, filt, out=out, roi=((x0, y0, z0), (x1, y1, z1)))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        lin = (idx[:, 0] * 512 + idx[:, 1]) * 512 + idx[:, 2]      # linear voxel numbers
        ref = oracle.correlate_points(src, w, lin, 0.0, 1.0)
        err = np.max(np.abs(got[idx[:, 0], idx[:, 1], idx[:, 2]] - ref)) / oracle.error_scale(w, 1.0)
        assert err <= 1e-5, err
        assert np.all(got[outside[:, 0], outside[:, 1], outside[:, 2]] == -3.0)
