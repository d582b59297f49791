"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped tap, a flipped
kernel, a wrong anchor, zero padding instead of clamping, a wrong mapping, a transposed
axis, a missing boundary fold in the adjoint) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rnd_vol(seed, shape, lo=-1.0, hi=1.0):
    return synth.uniform(seed, shape, lo, hi)


def rnd_w(seed, k):
    return synth.normal(seed, (k, k, k), 0.0, 1.0).astype(np.float64)


# ---------------------------------------------------------------------- identity, constant

@pytest.mark.parametrize("k", [1, 3, 5])
def test_identity_kernel_reproduces_input(k):
    x = rnd_vol(1, (5, 6, 7))
    w = np.zeros((k, k, k))
    w[k // 2, k // 2, k // 2] = 1.0
    y = oracle.correlate(x, w)
    assert np.array_equal(y, x.astype(np.float64))


@pytest.mark.parametrize("fmt,bits", [(synth.U8, 8), (synth.U16, 16)])
def test_identity_kernel_integer_mapping(fmt, bits):
    q = (synth.uniform(2, (4, 5, 6)) * (2 ** bits - 1)).astype(synth.NP_DTYPE[fmt])
    q.flat[0] = 0
    q.flat[1] = 2 ** bits - 1
    w = np.zeros((3, 3, 3))
    w[1, 1, 1] = 1.0
    lo, hi = -2.0, 6.0
    y = oracle.correlate(q, w, lo, hi)
    expect = lo + (hi - lo) * q.astype(np.float64) / (2 ** bits - 1)
    assert np.allclose(y, expect, rtol=0, atol=1e-15)
    assert y.flat[0] == lo and y.flat[1] == hi     # code 0 <-> lo, max code <-> hi


def test_constant_volume():
    c = 0.7314
    x = np.full((6, 5, 9), c, np.float32)
    g = oracle.gaussian_weights(5, 1.5)
    y = oracle.correlate(x, g)
    assert np.max(np.abs(y - float(np.float32(c)) * g.sum())) < 1e-12
    assert abs(g.sum() - 1.0) < 1e-6
    w = rnd_w(3, 3)
    y = oracle.correlate(x, w)
    assert np.max(np.abs(y - float(np.float32(c)) * w.sum())) < 1e-12


# ---------------------------------------------------------------------- linearity

def test_linear_in_kernel():
    x = rnd_vol(4, (7, 8, 9))
    w1, w2 = rnd_w(5, 3), rnd_w(6, 3)
    a, b = 0.37, -1.9
    lhs = oracle.correlate(x, a * w1 + b * w2)
    rhs = a * oracle.correlate(x, w1) + b * oracle.correlate(x, w2)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_linear_in_input():
    # small integers so that 3*x1 - 2*x2 is exact in float32
    x1 = np.floor(rnd_vol(7, (6, 7, 8), 0, 50)).astype(np.float32)
    x2 = np.floor(rnd_vol(8, (6, 7, 8), 0, 50)).astype(np.float32)
    w = rnd_w(9, 5)
    lhs = oracle.correlate((3 * x1 - 2 * x2).astype(np.float32), w)
    rhs = 3 * oracle.correlate(x1, w) - 2 * oracle.correlate(x2, w)
    assert np.max(np.abs(lhs - rhs)) < 1e-10


# ---------------------------------------------------------------------- separable = 3 passes

def _pass_1d(v, g, axis):
    """1-D clamp-to-edge correlation along one axis, written independently of the oracle."""
    r = (len(g) - 1) // 2
    pad = [(0, 0)] * v.ndim
    pad[axis] = (r, r)
    vp = np.pad(v, pad, mode="edge")
    out = np.zeros_like(v)
    n = v.shape[axis]
    for i, gi in enumerate(g):
        sl = [slice(None)] * v.ndim
        sl[axis] = slice(i, i + n)
        out += float(gi) * vp[tuple(sl)]
    return out


@pytest.mark.parametrize("k,sigma", [(3, 1.0), (5, 1.5), (7, 7 / 3)])
def test_separable_gaussian_equals_three_passes(k, sigma):
    x = rnd_vol(10, (9, 6, 11), 0, 1)
    g = oracle.gaussian_1d(k, sigma)
    y = oracle.correlate(x, oracle.separable_weights(g, g, g))
    t = x.astype(np.float64)
    for axis in (2, 1, 0):      # x, then y, then z
        t = _pass_1d(t, g, axis)
    assert np.max(np.abs(y - t)) < 1e-12


def test_separable_distinct_axes_orientation():
    # different 1-D profiles per axis pin which weight index runs along which axis
    x = rnd_vol(11, (5, 6, 7))
    gx = np.array([0.1, 0.5, 0.2], np.float32)
    gy = np.array([0.3, -0.4, 0.9], np.float32)
    gz = np.array([-0.6, 0.25, 0.05], np.float32)
    y = oracle.correlate(x, oracle.separable_weights(gx, gy, gz))
    t = _pass_1d(_pass_1d(_pass_1d(x.astype(np.float64), gx, 2), gy, 1), gz, 0)
    assert np.max(np.abs(y - t)) < 1e-12


# ---------------------------------------------------------------------- library special cases

@pytest.mark.parametrize("k", [1, 3, 5])
def test_matches_scipy_nearest(k):
    ndimage = pytest.importorskip("scipy.ndimage")
    x = rnd_vol(12 + k, (6, 7, 5))
    w = rnd_w(20 + k, k)
    ref = ndimage.correlate(x.astype(np.float64), w, mode="nearest")
    assert np.max(np.abs(oracle.correlate(x, w) - ref)) < 1e-12


def test_matches_torch_replicate_conv3d():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    x = rnd_vol(30, (5, 8, 6))
    w = rnd_w(31, 3)
    xt = torch.from_numpy(x.astype(np.float64))[None, None]
    ref = F.conv3d(F.pad(xt, (1, 1, 1, 1, 1, 1), mode="replicate"),
                   torch.from_numpy(w)[None, None])[0, 0].numpy()
    assert np.max(np.abs(oracle.correlate(x, w) - ref)) < 1e-12


# ---------------------------------------------------------------------- hand-derived closed forms

def test_hot_voxel_gives_flipped_footprint():
    x = np.zeros((7, 7, 7), np.float32)
    p = (3, 3, 3)          # (z, y, x)
    x[p] = 1.0
    w = rnd_w(40, 3)
    y = oracle.correlate(x, w)
    # y(i) = sum_d w[d] x(i+d-r) = w[p - i + r] for |p - i| <= r, else 0
    for iz in range(7):
        for iy in range(7):
            for ix in range(7):
                dz, dy, dx = p[0] - iz + 1, p[1] - iy + 1, p[2] - ix + 1
                if 0 <= dz < 3 and 0 <= dy < 3 and 0 <= dx < 3:
                    assert y[iz, iy, ix] == w[dz, dy, dx]
                else:
                    assert y[iz, iy, ix] == 0.0


def test_ramp_interior_unchanged_faces_shifted():
    z, yy, xx = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    v = (xx + 4 * yy + 16 * z).astype(np.float32)
    g = oracle.gaussian_1d(3, 1.0)
    y = oracle.correlate(v, oracle.separable_weights(g, g, g))
    # per axis the filter maps coordinate i to E[clamp(i + A)], A in {-1,0,1} with
    # probabilities g: interior i -> i, i = 0 -> g[2] (only the +1 tap moves), i = 3 -> 3 - g[0]
    g0, g2 = float(g[0]), float(g[2])
    s = float(np.sum(g.astype(np.float64)))

    def m(i):
        if i == 0:
            return (0 * (g0 + float(g[1])) + 1 * g2)
        if i == 3:
            return (2 * g0 + 3 * (float(g[1]) + g2))
        return i * s
    for iz in range(4):
        for iy in range(4):
            for ix in range(4):
                expect = (m(ix) + 4 * m(iy) + 16 * m(iz)) * s * s
                assert abs(y[iz, iy, ix] - expect) < 1e-12
    assert abs(y[1, 2, 1] - (1 + 8 + 16)) < 1e-6           # interior: unchanged


def _read_golden(name):
    spec = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            spec[key] = vals
    return spec


def test_golden_fillrange_then_gaussian_blur():
    spec = _read_golden("fillrange_teaser_64.txt")
    nx, ny, nz = (int(v) for v in spec["dims"])
    assert spec["format"] == ["uint8"]
    lo, hi = (float(v) for v in spec["range"])
    x0, y0, z0, x1, y1, z1 = (int(v) for v in spec["fillrange"])
    fill = float(spec["fillvalue"][0])
    code = int(round((fill - lo) / (hi - lo) * 255))
    vol = np.zeros((nz, ny, nx), np.uint8)
    vol[z0:z1, y0:y1, x0:x1] = code
    kind, k, sigma = spec["filter"][0], int(spec["filter"][1]), float(spec["filter"][2])
    assert kind == "gaussian" and k == 3
    y = oracle.correlate(vol, oracle.gaussian_weights(k, sigma), lo, hi)
    # closed form: exact sampled weights g = (e, 1, e)/(1 + 2e), e = exp(-1/(2 sigma^2));
    # per axis the fraction of the kernel landing inside [first, last) is
    #   0 at distance >= 2 outside, e/(1+2e) on the border voxel, 1 - e/(1+2e) on the
    #   first/last filled voxel, 1 deeper inside.
    e = math.exp(-1.0 / (2 * sigma * sigma))
    g0 = e / (1 + 2 * e)

    def frac(i, a, b):
        if i < a - 1 or i > b:
            return 0.0
        if i == a - 1 or i == b:
            return g0
        if i == a or i == b - 1:
            return 1.0 - g0
        return 1.0

    pts = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (32, 32, 32), (0, 32, 32), (1, 32, 32),
           (63, 63, 63), (62, 62, 62), (63, 1, 32), (61, 62, 0)]
    for (ix, iy, iz) in pts:
        expect = fill * frac(ix, x0, x1) * frac(iy, y0, y1) * frac(iz, z0, z1)
        assert abs(y[iz, iy, ix] - expect) < 2e-7, (ix, iy, iz)


# ---------------------------------------------------------------------- Gaussian construction

@pytest.mark.parametrize("k,sigma", [(3, 1.0), (5, 1.5), (7, 7 / 3), (9, 3.0)])
def test_gaussian_1d_properties(k, sigma):
    g = oracle.gaussian_1d(k, sigma).astype(np.float64)
    r = k // 2
    assert abs(g.sum() - 1.0) < 1e-6
    assert np.array_equal(g, g[::-1])
    for d in range(1, r + 1):
        assert abs(g[r + d] / g[r] - math.exp(-d * d / (2 * sigma * sigma))) < 1e-6


# ---------------------------------------------------------------------- quantisation

def test_quantize_ties_and_clamps():
    v = np.array([2.5, 3.5, -1.0, 300.0, 127.2, 127.7, 0.0, 255.0]) / 255.0
    t, q, tie = oracle.quantize(v, oracle.U8, 0.0, 1.0)
    assert list(q) == [2, 4, 0, 255, 127, 128, 0, 255]
    assert list(tie) == [True, True, False, False, False, False, False, False]
    t, q, tie = oracle.quantize(np.array([0.5]), oracle.U16, 0.0, 1.0)
    assert q[0] == round(0.5 * 65535)   # 32767.5 -> 32768 (even)
    assert tie[0]


# ---------------------------------------------------------------------- points == full

def test_points_match_full_volume():
    x = rnd_vol(50, (6, 5, 7))
    w = rnd_w(51, 5)
    full = oracle.correlate(x, w)
    idx = np.arange(x.size)
    pts = oracle.correlate_points(x, w, idx)
    assert np.array_equal(pts, full.ravel())


# ---------------------------------------------------------------------- gradients

def test_adjoint_dot_product():
    x = rnd_vol(60, (6, 7, 5))
    yv = rnd_vol(61, (6, 7, 5)).astype(np.float64)
    w = rnd_w(62, 5)
    cx = oracle.correlate(x, w)
    gx, gw = oracle.correlate_backward(x, yv, w)
    assert abs(np.sum(cx * yv) - np.sum(x.astype(np.float64) * gx)) < 1e-10
    # gw[d] = <C_{e_d} x, y>
    for d in [0, 17, 62, 124]:
        e = np.zeros(125)
        e[d] = 1.0
        assert abs(np.sum(oracle.correlate(x, e) * yv) - gw.ravel()[d]) < 1e-11


def test_backward_input_points_match_scatter():
    gy = rnd_vol(63, (4, 6, 5)).astype(np.float64)
    x = rnd_vol(64, (4, 6, 5))
    w = rnd_w(65, 5)             # k larger than one axis: several taps fold on a face
    gx, _ = oracle.correlate_backward(x, gy, w, need_gw=False)
    pts = oracle.backward_input_points(gy, w, np.arange(gy.size))
    assert np.max(np.abs(pts - gx.ravel())) < 1e-12


def test_gradients_match_central_differences():
    x = rnd_vol(70, (5, 6, 7), 0, 1)
    target = rnd_vol(71, (5, 6, 7), 0, 1).astype(np.float64)
    w = rnd_w(72, 3) * 0.1
    n = x.size

    def loss(wv, xv):
        return float(np.mean((oracle.correlate(xv, wv) - target) ** 2))

    y = oracle.correlate(x, w)
    gy = 2.0 * (y - target) / n
    gx, gw = oracle.correlate_backward(x, gy, w)
    h = 1e-3
    for d in [0, 4, 13, 26]:
        e = np.zeros(27)
        e[d] = h
        fd = (loss(w + e.reshape(3, 3, 3), x) - loss(w - e.reshape(3, 3, 3), x)) / (2 * h)
        assert abs(fd - gw.ravel()[d]) < 1e-9
    # input gradient on float32-exact perturbations (h a power of two)
    hx = 2.0 ** -10
    for j in [0, 37, n - 1]:
        xp = x.copy().ravel()
        xm = x.copy().ravel()
        xp[j] += np.float32(hx)
        xm[j] -= np.float32(hx)
        fd = (loss(w, xp.reshape(x.shape)) - loss(w, xm.reshape(x.shape))) / (2 * hx)
        assert abs(fd - gx.ravel()[j]) < 1e-9


def test_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    x = rnd_vol(80, (6, 5, 7))
    gy = rnd_vol(81, (6, 5, 7)).astype(np.float64)
    w = rnd_w(82, 5)
    xt = torch.from_numpy(x.astype(np.float64))[None, None].requires_grad_(True)
    wt = torch.from_numpy(w)[None, None].requires_grad_(True)
    y = F.conv3d(F.pad(xt, (2,) * 6, mode="replicate"), wt)
    y.backward(torch.from_numpy(gy)[None, None])
    gx, gw = oracle.correlate_backward(x, gy, w)
    assert np.max(np.abs(gx - xt.grad[0, 0].numpy())) < 1e-11
    assert np.max(np.abs(gw - wt.grad[0, 0].numpy())) < 1e-11


# ---------------------------------------------------------------------- a planted mistake

def test_planted_zero_padding_is_caught():
    """The scipy pin distinguishes clamp-to-edge from zero padding (mode='constant')."""
    ndimage = pytest.importorskip("scipy.ndimage")
    x = rnd_vol(90, (5, 5, 5), 0.5, 1.0)
    w = rnd_w(91, 3)
    wrong = ndimage.correlate(x.astype(np.float64), w, mode="constant")
    assert np.max(np.abs(oracle.correlate(x, w) - wrong)) > 1e-3


# ---------------------------------------------------------------------- BrickDecompose

BRICK_CASES = [((7, 5, 6), (3, 2, 4), 0), ((7, 5, 6), (3, 2, 4), 1), ((9, 4, 5), (4, 4, 4), 2),
               ((3, 3, 3), (8, 8, 8), 3), ((5, 6, 4), (1, 1, 1), 1)]


def brick_origins(shape, brick):
    nz, ny, nx = shape
    bx, by, bz = brick
    return [(ox, oy, oz) for oz in range(0, nz, bz) for oy in range(0, ny, by)
            for ox in range(0, nx, bx)]


@pytest.mark.parametrize("shape,brick,ghost", BRICK_CASES)
def test_bricks_match_edge_padded_slices(shape, brick, ghost):
    """Against numpy's own clamp-to-edge padding: brick = pad(src, ghost, 'edge') sliced at
    the brick's origin with the brick's stored size."""
    src = rnd_vol(100, shape)
    pad = np.pad(src, ghost, mode="edge")
    bricks = oracle.brick_decompose(src, brick, ghost)
    origins = brick_origins(shape, brick)
    assert len(bricks) == len(origins)
    nz, ny, nx = shape
    bx, by, bz = brick
    for b, (ox, oy, oz) in zip(bricks, origins):
        sx, sy, sz = min(bx, nx - ox), min(by, ny - oy), min(bz, nz - oz)
        assert b.shape == (sz + 2 * ghost, sy + 2 * ghost, sx + 2 * ghost)
        assert np.array_equal(b, pad[oz:oz + sz + 2 * ghost, oy:oy + sy + 2 * ghost,
                                     ox:ox + sx + 2 * ghost])


@pytest.mark.parametrize("shape,brick,ghost", BRICK_CASES)
def test_brick_interiors_tile_the_volume(shape, brick, ghost):
    """The interiors reassemble the volume exactly, each voxel once."""
    src = rnd_vol(101, shape)
    out = np.full(shape, np.nan)
    g = ghost
    for b, (ox, oy, oz) in zip(oracle.brick_decompose(src, brick, ghost), brick_origins(shape, brick)):
        inner = b[g:b.shape[0] - g, g:b.shape[1] - g, g:b.shape[2] - g]
        sl = (slice(oz, oz + inner.shape[0]), slice(oy, oy + inner.shape[1]), slice(ox, ox + inner.shape[2]))
        assert np.isnan(out[sl]).all()
        out[sl] = inner
    assert np.array_equal(out, src)


def test_brick_ghosts_hold_neighbours_and_repeat_faces():
    src = rnd_vol(102, (6, 6, 8))
    g = 2
    bricks = oracle.brick_decompose(src, (4, 6, 6), g)     # two bricks along x
    left, right = bricks
    # the left brick's +x ghost columns are the right brick's first interior columns
    assert np.array_equal(left[:, :, -g:], right[:, :, g:2 * g])
    assert np.array_equal(right[:, :, :g], left[:, :, -2 * g:-g])
    # beyond the -x face the ghosts repeat the face voxel; likewise in y and z
    for c in range(g):
        assert np.array_equal(left[:, :, c], left[:, :, g])
        assert np.array_equal(left[:, c, :], left[:, g, :])
        assert np.array_equal(left[c], left[g])


# ---------------------------------------------------------------------- CLAHE-3D

def u8_vol(seed, shape):
    return synth.quantize(synth.uniform(seed, shape), synth.U8)


def test_clahe_single_brick_without_clip_is_histogram_equalisation():
    """One brick, no clip limit: the textbook global histogram equalisation of the codes."""
    v = u8_vol(110, (10, 12, 14))
    out, t, luts = oracle.clahe3d(v, (1, 1, 1), 0.0)
    n = v.size
    cdf = np.cumsum(np.bincount(v.ravel(), minlength=256))
    lut = np.minimum((255 * cdf + n // 2) // n, 255)
    assert np.array_equal(luts[0, 0, 0], lut)
    assert np.array_equal(out, lut[v])


def test_clahe_hand_computed_brick_at_the_minimum_limit():
    """A 2 x 2 x 2 brick of code 10 (N = 8) under clip 1: the limit floor(1 * 8 / 256) = 0
    is raised to 1 count, so h[10] = 8 keeps 1 and the excess 7 goes back one count each to
    bins 0, 36, 72, ..., 216 (step 256 // 7 = 36).  Then cdf[10] = h[0] + h[10] = 2 and
    lut[10] = (255 * 2 + 8 // 2) // 8 = 64, which every voxel takes.  Without a clip limit
    cdf[10] = 8 and the code maps to 255."""
    v = np.full((2, 2, 2), 10, np.uint8)
    out, t, luts = oracle.clahe3d(v, (1, 1, 1), 1.0)
    assert np.all(out == 64) and np.all(t == 64.0)
    assert luts[0, 0, 0, 10] == 64
    assert luts[0, 0, 0].tolist()[:37] == [32] * 10 + [64] * 26 + [96]   # bins 0, 10 and 36
    out, _, _ = oracle.clahe3d(v, (1, 1, 1), 0.0)
    assert np.all(out == 255)


def test_clahe_exact_ties_round_to_even():
    """Blends of 2 x 2 bricks of 4 x 4 voxels weigh the mappings by multiples of 1/16, so
    some land exactly on k + 0.5; the code is then the even neighbour (and otherwise the
    nearest integer)."""
    v = np.random.default_rng(1).integers(0, 256, size=(1, 8, 8)).astype(np.uint8)
    out, t, _ = oracle.clahe3d(v, (2, 2, 1), 0.0)
    ties = (t - np.floor(t)) == 0.5
    assert ties.sum() >= 3
    assert np.all(out[ties] % 2 == 0)
    assert np.all(np.abs(out[ties].astype(np.float64) - t[ties]) == 0.5)
    assert np.array_equal(out, np.rint(t).astype(np.uint8))


@pytest.mark.parametrize("clip", [0.5, 1.0, 3.0, 40.0])
def test_clahe_clip_conserves_counts_and_limits_contrast(clip):
    v = synth.quantize(synth.blobs(111, (12, 12, 12), nblobs=3, sigma=(2.0, 5.0)), synth.U8)
    n = v.size
    _, _, luts = oracle.clahe3d(v, (1, 1, 1), clip)
    lut = luts[0, 0, 0].astype(np.int64)
    assert lut[255] == 255                      # the redistributed counts still sum to N
    assert np.all(np.diff(lut) >= 0)            # a mapping that keeps the order of codes
    limit = max(1, int(np.floor(clip * n / 256)))
    # one code adds at most limit + ceil(excess/256) + 1 counts: its contrast is capped
    cap = (limit + (n // 256) + 2) * 255 / n + 1
    assert np.max(np.diff(lut)) <= cap


def test_clahe_brick_centres_take_their_own_mapping():
    """With odd brick sizes a voxel at a brick centre has interpolation weights 0/1, so it
    maps through its own brick's mapping exactly."""
    v = u8_vol(112, (10, 15, 20))             # bricks 5 x 5 x 5 for nb = (4, 3, 2)
    out, _, luts = oracle.clahe3d(v, (4, 3, 2), 2.0)
    for bz in range(2):
        for by in range(3):
            for bx in range(4):
                x, y, z = 5 * bx + 2, 5 * by + 2, 5 * bz + 2
                assert out[z, y, x] == luts[bz, by, bx, v[z, y, x]]


def test_clahe_blend_is_scipy_trilinear_interpolation():
    """Between the centres the result is the linear interpolation (edge-clamped) of the
    bricks' mappings at the voxel's brick coordinate, as scipy's map_coordinates computes."""
    ndimage = pytest.importorskip("scipy.ndimage")
    v = u8_vol(113, (8, 12, 16))
    nb = (4, 3, 2)
    _, t, luts = oracle.clahe3d(v, nb, 1.5)
    nz, ny, nx = v.shape
    s = (nx // nb[0], ny // nb[1], nz // nb[2])
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [(zz + 0.5) / s[2] - 0.5, (yy + 0.5) / s[1] - 0.5, (xx + 0.5) / s[0] - 0.5]
    ref = np.empty(v.shape)
    for q in np.unique(v):
        m = v == q
        grid = luts[..., q].astype(np.float64)
        ref[m] = ndimage.map_coordinates(grid, [c[m] for c in coords], order=1, mode="nearest")
    assert np.max(np.abs(ref - t)) < 1e-9


def test_clahe_constant_volume_stays_constant():
    v = np.full((8, 8, 8), 77, dtype=np.uint8)
    out, _, _ = oracle.clahe3d(v, (2, 2, 2), 2.0)
    assert np.all(out == out[0, 0, 0])


# ---------------------------------------------------------------------- headless Render

def render_uniform(value, lut, step=0.5, termination=2.0, size=(16, 12), eye=(4, 4, -20)):
    v = np.full((8, 8, 8), value, np.float32)
    return oracle.render(v, 0.0, 1.0, size[0], size[1], eye, (4, 4, 4), (0, 1, 0), 0.5, step,
                         termination, (0.1, 0.2, 0.3, 0.4), lut)


def test_render_transparent_volume_shows_the_background():
    img = render_uniform(0.5, [[1, 1, 1, 0], [1, 1, 1, 0]])
    assert np.allclose(img, np.array([0.1, 0.2, 0.3, 0.4]), atol=0, rtol=0)


@pytest.mark.parametrize("step", [0.5, 0.25, 1.0])
def test_render_uniform_slab_follows_beer_lambert(step):
    """The centre ray crosses 8 voxel lengths of a uniform medium of per-voxel opacity a:
    accumulated opacity 1 - (1 - a)^8 for any step dividing the path, colour c times it,
    then the background behind."""
    a = 0.1
    # pixel (7, 5) of a 15 x 11 image looks along the axis, through z = 0 .. 8
    img = render_uniform(0.5, [[0.8, 0.4, 0.2, a], [0.8, 0.4, 0.2, a]], step=step, size=(15, 11))
    A = 1 - (1 - a) ** 8
    px = img[5, 7]
    assert abs(px[3] - (A + (1 - A) * 0.4)) < 1e-12
    assert np.allclose(px[:3], np.array([0.8, 0.4, 0.2]) * A + (1 - A) * np.array([0.1, 0.2, 0.3]), atol=1e-12)


def test_render_stops_at_the_termination_opacity():
    a, step = 0.1, 0.5
    img = render_uniform(0.5, [[1, 1, 1, a], [1, 1, 1, a]], step=step, termination=0.3, size=(15, 11))
    ac = 1 - (1 - a) ** step
    k = int(np.ceil(np.log(1 - 0.3) / np.log(1 - ac)))
    A = 1 - (1 - ac) ** k
    assert abs(img[5, 7, 3] - (A + (1 - A) * 0.4)) < 1e-12


def test_render_table_is_blended_linearly():
    """Value 0.25 between two table entries: colour 0.75 c0 + 0.25 c1."""
    lut = [[1.0, 0.0, 0.0, 0.5], [0.0, 0.0, 1.0, 0.5]]
    img = render_uniform(0.25, lut, size=(15, 11))
    A = 1 - 0.5 ** 8
    px = img[5, 7]
    assert np.allclose(px[:3], np.array([0.75, 0.0, 0.25]) * A + (1 - A) * np.array([0.1, 0.2, 0.3]), atol=1e-12)


def test_render_camera_orientation():
    """Looking along +z with +y up, the right edge of the image is towards -x: an opaque
    slab at low x appears in the right half, one at high y in the top half."""
    v = np.zeros((8, 8, 8), np.float32)
    v[:, :, :3] = 1.0                     # low x
    lut = [[0, 0, 0, 0], [1, 1, 1, 1]]
    img = oracle.render(v, 0.0, 1.0, 31, 31, (4, 4, -20), (4, 4, 4), (0, 1, 0), 0.5, 0.25, 2.0,
                        (0, 0, 0, 0), lut)
    assert img[15, 25, 3] > 0.5 and img[15, 5, 3] < 0.5
    v = np.zeros((8, 8, 8), np.float32)
    v[:, 5:, :] = 1.0                     # high y
    img = oracle.render(v, 0.0, 1.0, 31, 31, (4, 4, -20), (4, 4, 4), (0, 1, 0), 0.5, 0.25, 2.0,
                        (0, 0, 0, 0), lut)
    assert img[5, 15, 3] > 0.5 and img[25, 15, 3] < 0.5


def test_render_miss_rays_see_background():
    img = render_uniform(0.5, [[1, 1, 1, 1], [1, 1, 1, 1]], size=(64, 48))
    assert np.allclose(img[0, 0], [0.1, 0.2, 0.3, 0.4])


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("step", [0.5, 0.25])
def test_render_samples_ramps_at_voxel_centres(axis, step):
    """Trilinear sampling with voxel centres at i + 0.5: a volume that rises by 1/8 per voxel
    along one axis is read along the ray as clamp(p - 0.5, 0, 7) / 8, p the ray's coordinate
    on that axis (exact for a linear ramp; clamped beyond the outer centres).  With a table
    whose colour equals the value and whose opacity is a constant a, the centre pixel is
    ac * sum_k (1 - ac)^k s_k + (1 - ac)^K bg, ac = 1 - (1 - a)^step.  An axis mix-up or a
    half-voxel shift in the sampler changes the result."""
    n, a = 8, 0.2
    ramp = np.arange(n, dtype=np.float64) / 8.0
    shape = [1, 1, 1]
    shape[2 - axis] = n                               # (z, y, x) array order
    v = np.broadcast_to(ramp.reshape(shape), (n, n, n)).astype(np.float32).copy()
    eye = np.array([3.2, 5.9, -20.0])
    lut = [[0, 0, 0, a], [1, 1, 1, a]]
    bg = np.array([0.1, 0.2, 0.3, 0.4])
    # pixel (7, 5) of a 15 x 11 image is the ray along +z through (3.2, 5.9)
    px = oracle.render(v, 0.0, 1.0, 15, 11, eye, (3.2, 5.9, 4.0), (0, 1, 0), 0.5, step, 2.0,
                       bg, lut)[5, 7]
    zs = (np.arange(int(round(n / step))) + 0.5) * step  # sample depths inside [0, 8)
    p = zs if axis == 2 else np.full_like(zs, eye[axis])
    s = np.clip(p - 0.5, 0.0, n - 1.0) / 8.0
    ac = 1.0 - (1.0 - a) ** step
    trans = (1.0 - ac) ** np.arange(len(zs))
    C = ac * np.sum(trans * s)
    A = 1.0 - (1.0 - ac) ** len(zs)
    assert np.allclose(px[:3], C + (1.0 - A) * bg[:3], atol=1e-12, rtol=0)
    assert abs(px[3] - (A + (1.0 - A) * bg[3])) < 1e-12


def test_render_silhouette_of_a_cube_keeps_square_pixels():
    """Pinhole projection of an opaque 8^3 cube seen face-on from 20 voxels in front of it:
    the ray through pixel (px, py) has direction ~ (-sx, sy, 1) with
    sx = (2 (px + 0.5) / W - 1) tan(fovy/2) W/H and sy = (1 - 2 (py + 0.5) / H) tan(fovy/2),
    and enters the front face iff |sx| <= 4/20 and |sy| <= 4/20.  With tan(fovy/2) = 0.41
    on a 40 x 20 image that is columns 15..24 and rows 5..14: a square silhouette, since
    the horizontal angle per pixel equals the vertical one."""
    import math
    v = np.ones((8, 8, 8), np.float32)
    fovy = 2 * math.atan(0.41)
    img = oracle.render(v, 0.0, 1.0, 40, 20, (4, 4, -20), (4, 4, 4), (0, 1, 0), fovy, 0.5, 2.0,
                        (0, 0, 0, 0), [[1, 1, 1, 1], [1, 1, 1, 1]])
    want = np.zeros((20, 40))
    want[5:15, 15:25] = 1.0
    assert np.array_equal(img[..., 3], want)


def test_laplacian_stencil_is_exact_on_quadratics():
    """The 7-point Laplacian is the exact Laplacian of any quadratic: on
    f = x^2 + 2 y^2 + 3 z^2 + x y - 4 z + 5 it gives 2 + 4 + 6 = 12 at every interior voxel,
    and 0 on any linear field; it has 7 non-zero taps summing to 0."""
    w = oracle.laplacian_3()
    assert np.count_nonzero(w) == 7 and w.sum() == 0.0
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(8.0), np.arange(7.0), indexing="ij")
    f = x ** 2 + 2 * y ** 2 + 3 * z ** 2 + x * y - 4 * z + 5
    out = oracle.correlate(f.astype(np.float32), w)
    assert np.allclose(out[1:-1, 1:-1, 1:-1], 12.0, rtol=0, atol=1e-9)
    lin = (2 * x - 3 * y + 0.5 * z + 1).astype(np.float32)
    assert np.allclose(oracle.correlate(lin, w)[1:-1, 1:-1, 1:-1], 0.0, rtol=0, atol=1e-9)
