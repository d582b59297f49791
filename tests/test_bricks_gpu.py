"""GPU parity of BrickDecompose (vktBrickDecomposeSV): every brick, ghost cells included,
bit-exact against the oracle's decomposition, for every storage format, brick sizes that do
and do not divide the volume (and exceed it), and ghost widths 0 to beyond a brick."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 800


def volume(fmt, shape, seed):
    if fmt == synth.F32:
        return synth.uniform(seed, shape, -3.0, 3.0)
    return synth.quantize(synth.uniform(seed, shape), fmt)


@pytest.mark.parametrize("fmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("shape,brick,ghost", [
    ((40, 37, 70), (16, 16, 16), 0),
    ((40, 37, 70), (16, 16, 16), 2),
    ((33, 20, 65), (64, 8, 11), 3),      # x brick wider than the volume
    ((9, 10, 11), (4, 3, 2), 5),         # ghost wider than a brick
    ((1, 1, 1), (1, 1, 1), 1),
    ((20, 18, 66), (33, 7, 5), 1),       # rows of odd length: words straddle brick rows
    ((3, 4, 1500), (700, 2, 2), 1),      # long rows: a row's blocks outnumber a warp's lanes
    ((20, 18, 64), (16, 8, 8), 0),       # 16-byte aligned spans: block copies
    ((12, 10, 48), (16, 5, 6), 0),
])
def test_bricks_match_oracle(fmt, shape, brick, ghost):
    src = volume(fmt, shape, SEED + sum(shape) + ghost)
    got = vkt.brick_decompose(torch.from_numpy(src).cuda(), brick, ghost)
    torch.cuda.synchronize()
    vkt.synchronize()
    ref = oracle.brick_decompose(src, brick, ghost)
    assert len(got) == len(ref)
    for i, (g, r) in enumerate(zip(got, ref)):
        g = g.cpu().numpy()
        assert g.shape == r.shape, i
        assert np.array_equal(g.view(np.uint8), np.ascontiguousarray(r).view(np.uint8)), f"brick {i}"


@pytest.mark.parametrize("fmt,shape,brick,ghost", [
    (synth.U8, (37, 45, 64), (16, 16, 16), 2),    # faces on every axis, partial bricks in y, z
    (synth.U8, (20, 30, 80), (32, 10, 6), 4),     # the last brick along x is partial (16 wide)
    (synth.U8, (9, 40, 48), (16, 8, 4), 16),      # the widest ghost the 16-byte halo holds
    (synth.U16, (25, 19, 40), (8, 8, 8), 2),
    (synth.U16, (10, 12, 16), (8, 5, 4), 1),      # 20-byte rows: shifts of 2 bytes
    (synth.U16, (6, 7, 24), (8, 4, 3), 8),
    (synth.F32, (21, 22, 28), (12, 8, 8), 3),     # partial last brick along x
    (synth.F32, (13, 9, 32), (4, 4, 5), 4),
    (synth.F32, (8, 6, 16), (4, 3, 2), 1),
    (synth.U8, (10, 12, 16), (32, 4, 4), 2),      # bricks wider than the volume: the box
    (synth.U16, (6, 9, 8), (16, 16, 3), 3),       # reaches past it (zero-filled, never read)
    (synth.F32, (5, 7, 4), (8, 8, 8), 1),
])
def test_plane_image_kernel(fmt, shape, brick, ghost, capfd):
    """Ghost cells on a source a tensor map describes, brick widths of whole 16-byte blocks
    and brick rows of whole words take the plane-image kernel (one box per brick plane, one
    funnel shift per word, voxel-by-voxel words at the x faces): bit-exact against the
    oracle for every format, ghost widths up to the 16-byte halo, partial bricks and
    clamping on every face."""
    src = volume(fmt, shape, SEED + 31 + sum(shape) + ghost)
    capfd.readouterr()
    with vkt.policy(debug=vkt.DEBUG_LOG):
        got = vkt.brick_decompose(torch.from_numpy(src).cuda(), brick, ghost)
        torch.cuda.synchronize()
    err = capfd.readouterr().err
    assert " planes launches=" in err, err
    vkt.synchronize()
    ref = oracle.brick_decompose(src, brick, ghost)
    assert len(got) == len(ref)
    for i, (g, r) in enumerate(zip(got, ref)):
        g = g.cpu().numpy()
        assert g.shape == r.shape, i
        assert np.array_equal(g.view(np.uint8), np.ascontiguousarray(r).view(np.uint8)), f"brick {i}"


def test_bricks_of_the_512_volume_reassemble_it():
    """The 512^3 uint8 CT-like volume in 64^3 bricks with 2 ghost cells (the halo a 5^3
    filter needs): interiors reassemble the volume, ghosts match their neighbours."""
    src = synth.volume("blobs", synth.U8, (512, 512, 512), synth.BASE_SEED + 1)
    s = torch.from_numpy(src).cuda()
    g = 2
    bricks = vkt.brick_decompose(s, (64, 64, 64), g)
    torch.cuda.synchronize()
    assert len(bricks) == 512
    inner = torch.empty_like(s)
    for i, b in enumerate(bricks):
        kz, ky, kx = i // 64, (i // 8) % 8, i % 8
        inner[kz * 64:(kz + 1) * 64, ky * 64:(ky + 1) * 64, kx * 64:(kx + 1) * 64] = b[g:-g, g:-g, g:-g]
    assert torch.equal(inner, s)
    # ghosts of an interior brick are the neighbouring voxels of the volume
    b = bricks[(3 * 8 + 4) * 8 + 5]
    assert torch.equal(b, s[3 * 64 - g:4 * 64 + g, 4 * 64 - g:5 * 64 + g, 5 * 64 - g:6 * 64 + g])


@pytest.mark.parametrize("fmt", [synth.U8, synth.U16, synth.F32])
def test_staged_and_plain_paths(fmt, capfd):
    """A 16-byte aligned source takes the staged kernel; the same voxels one element further
    into a buffer (not 16-byte aligned) take the plain one.  Both bit-exact."""
    shape, brick, ghost = (21, 30, 45), (16, 16, 8), 2
    src = volume(fmt, shape, SEED + 5)
    ref = oracle.brick_decompose(src, brick, ghost)
    t = torch.from_numpy(src).cuda()
    flat = torch.empty(t.numel() + 1, dtype=t.dtype, device="cuda")
    flat[1:] = t.reshape(-1)
    shifted = flat[1:].view(shape)
    for s, path in ((t, "staged"), (shifted, "plain")):
        capfd.readouterr()
        with vkt.policy(debug=vkt.DEBUG_LOG):
            got = vkt.brick_decompose(s, brick, ghost)
            torch.cuda.synchronize()
        err = capfd.readouterr().err
        assert f" {path} " in err, err
        for i, (g, r) in enumerate(zip(got, ref)):
            assert np.array_equal(g.cpu().numpy().view(np.uint8),
                                  np.ascontiguousarray(r).view(np.uint8)), f"{path} brick {i}"


def test_more_bricks_than_one_launch_takes():
    """4000 bricks of 1 x 1 x 2 voxels with a ghost cell: the bricks' pointers travel as
    launch parameters, 3968 per launch, so this call takes two launches."""
    shape = (20, 20, 20)
    src = volume(synth.U8, shape, SEED + 77)
    got = vkt.brick_decompose(torch.from_numpy(src).cuda(), (1, 1, 2), 1)
    torch.cuda.synchronize()
    ref = oracle.brick_decompose(src, (1, 1, 2), 1)
    assert len(got) == len(ref) == 4000
    g = torch.stack([t.reshape(-1) for t in got]).cpu().numpy()
    r = np.stack([np.ascontiguousarray(t).reshape(-1) for t in ref])
    assert np.array_equal(g, r)


@pytest.mark.parametrize("shape,brick,ghost,path", [((20, 18, 64), (16, 8, 8), 0, "staged blocks"),
                                                    ((20, 18, 64), (16, 8, 8), 1, "staged grid"),
                                                    ((20, 18, 72), (16, 8, 8), 0, "staged grid")])
def test_block_only_kernel_when_every_brick_is_aligned(shape, brick, ghost, path, capfd):
    """Without ghost cells, with 16-byte rows and brick widths (the last brick along x of
    the 72-wide volume is 8 bytes wide, so that one takes the general kernel), a call runs
    the kernel that holds only the block copies; results bit-exact either way."""
    src = volume(synth.U8, shape, SEED + 9)
    capfd.readouterr()
    with vkt.policy(debug=vkt.DEBUG_LOG):
        got = vkt.brick_decompose(torch.from_numpy(src).cuda(), brick, ghost)
        torch.cuda.synchronize()
    err = capfd.readouterr().err
    want = "staged blocks" if path == "staged blocks" else "staged launches"
    assert want in err, err
    for g, r in zip(got, oracle.brick_decompose(src, brick, ghost)):
        assert np.array_equal(g.cpu().numpy(), r)
