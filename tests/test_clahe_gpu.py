"""GPU parity of CLAHE-3D (vktClahe3DSV) against the FP64 oracle: codes equal except where the
oracle's blended value lies within 1e-3 of a rounding tie (there either neighbour is
accepted), for clipped and unclipped equalisation, brick grids with even and odd brick
sizes, and the paper's 256^3 size."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 900


def ct_like(shape, seed):
    nz, ny, nx = shape
    return synth.volume("blobs", synth.U8, (nx, ny, nz), seed)


def check(gpu, ref, t, what):
    frac = np.abs(t - np.floor(t) - 0.5)
    tie = frac < 1e-3
    bad = (gpu != ref) & ~tie
    assert not bad.any(), f"{what}: {int(bad.sum())} codes differ outside tie windows"
    near = np.abs(gpu[tie].astype(np.int64) - ref[tie].astype(np.int64))
    assert np.all(near <= 1), f"{what}: tie voxels off by more than one code"


@pytest.mark.parametrize("shape,bricks", [((64, 64, 64), (4, 4, 4)), ((48, 64, 96), (3, 2, 4)),
                                          ((30, 25, 35), (7, 5, 6)), ((16, 16, 16), (1, 1, 1)),
                                          ((24, 20, 36), (3, 2, 2))])
@pytest.mark.parametrize("clip", [0.0, 1.0, 2.0, 40.0])
def test_clahe_matches_oracle(shape, bricks, clip):
    v = ct_like(shape, SEED + sum(shape))
    clip = float(np.float32(clip))
    got = vkt.clahe3d(torch.from_numpy(v).cuda(), bricks, clip)
    torch.cuda.synchronize()
    vkt.synchronize()
    ref, t, _ = oracle.clahe3d(v, bricks, clip)
    check(got.cpu().numpy(), ref, t, f"{shape} bricks {bricks} clip {clip}")


@pytest.mark.parametrize("shape,bricks,vec,blend", [((64, 64, 64), (4, 4, 4), 16, "cells"),
                                                   ((24, 20, 36), (3, 2, 2), 4, "voxels"),
                                                   ((30, 25, 35), (7, 5, 6), 1, "voxels")])
def test_clahe_paths(shape, bricks, vec, blend, capfd):
    """Which histogram load width and which blend kernel a shape takes (each is covered by the
    parity cases above)."""
    v = torch.from_numpy(ct_like(shape, SEED)).cuda()
    capfd.readouterr()
    with vkt.policy(debug=vkt.DEBUG_LOG):
        vkt.clahe3d(v, bricks, 2.0)
        torch.cuda.synchronize()
    err = capfd.readouterr().err
    assert f"blend={blend}" in err and f"loads of {vec} bytes" in err, err


def test_clahe_paper_size_256():
    """The paper's case-study size, 256^3, in 8^3 bricks of 32^3 voxels, clip 2."""
    v = ct_like((256, 256, 256), SEED + 1)
    got = vkt.clahe3d(torch.from_numpy(v).cuda(), (8, 8, 8), 2.0)
    torch.cuda.synchronize()
    ref, t, _ = oracle.clahe3d(v, (8, 8, 8), 2.0)
    check(got.cpu().numpy(), ref, t, "256^3")


def test_clahe_rejects_bad_arguments():
    v = torch.from_numpy(ct_like((16, 16, 16), SEED)).cuda()
    with pytest.raises(vkt.VktError) as e:
        vkt.clahe3d(v, (3, 4, 4), 2.0)               # 3 bricks do not divide 16
    assert e.value.code == 1
    f = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(vkt.VktError) as e:
        vkt.clahe3d(f, (2, 2, 2), 2.0)               # float32 volumes are not supported
    assert e.value.code == 4
