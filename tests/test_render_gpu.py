"""GPU parity of the headless Render (vktRenderSV: ray marching with absorption and emission)
against the FP64 oracle: every pixel's RGBA within 2e-4, for uint8 / uint16 / float32
volumes, oblique and axis-aligned cameras, a camera inside the volume, early termination,
and ragged image sizes."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 1000
TOL = 2e-4

RAMP = np.array([[0.0, 0.0, 0.0, 0.0], [0.9, 0.5, 0.2, 0.02], [1.0, 0.9, 0.6, 0.15],
                 [1.0, 1.0, 1.0, 0.6]], dtype=np.float32)
RAINBOW = np.array([[0, 0, 1, 0.05], [0, 1, 1, 0.1], [0, 1, 0, 0.0], [1, 1, 0, 0.3], [1, 0, 0, 0.8]],
                   dtype=np.float32)


def volume(fmt, shape, seed):
    nz, ny, nx = shape
    if fmt == synth.F32:
        return synth.fourier(seed, (nx, ny, nz), nmodes=8).astype(np.float32)
    return synth.volume("blobs", fmt, (nx, ny, nz), seed)


CAMERAS = [
    dict(eye=(24.0, 20.0, -40.0), center=(24.0, 20.0, 16.0), up=(0.0, 1.0, 0.0), fovy=0.9),
    dict(eye=(-30.0, 55.0, 70.0), center=(20.0, 18.0, 14.0), up=(0.0, 1.0, 0.2), fovy=0.7),
    dict(eye=(20.0, 18.0, 14.0), center=(60.0, 10.0, 30.0), up=(0.0, 0.0, 1.0), fovy=1.4),  # inside
]


@pytest.mark.parametrize("fmt", [synth.U8, synth.U16, synth.F32])
@pytest.mark.parametrize("cam", range(len(CAMERAS)))
def test_render_matches_oracle(fmt, cam):
    shape = (32, 40, 48)
    v = volume(fmt, shape, SEED + fmt)
    lo, hi = (0.0, 1.0) if fmt != synth.F32 else (float(v.min()), float(v.max()))
    c = CAMERAS[cam]
    lut = RAMP if fmt != synth.F32 else RAINBOW
    w, h, step, term = 37, 29, 0.5, 2.0
    got = vkt.render(torch.from_numpy(v).cuda(), w, h, c["eye"], c["center"], c["up"], c["fovy"],
                     step, lut, termination=term, background=(0.1, 0.1, 0.2, 1.0), src_range=(lo, hi))
    torch.cuda.synchronize()
    vkt.synchronize()
    # the library takes float32 parameters: give the oracle the same values
    f32 = lambda x: [float(np.float32(t)) for t in x]
    ref = oracle.render(v, float(np.float32(lo)), float(np.float32(hi)), w, h, f32(c["eye"]),
                        f32(c["center"]), f32(c["up"]), float(np.float32(c["fovy"])), step, term,
                        (0.1, 0.1, 0.2, 1.0), lut)
    err = np.max(np.abs(got.cpu().numpy().astype(np.float64) - ref))
    assert err <= TOL, f"max |gpu - oracle| = {err:.2e}"


def test_render_early_termination_and_step():
    v = volume(synth.U8, (32, 40, 48), SEED + 7)
    c = CAMERAS[1]
    for step, term in ((0.25, 0.95), (1.0, 0.5), (0.7, 2.0)):
        got = vkt.render(torch.from_numpy(v).cuda(), 40, 30, c["eye"], c["center"], c["up"], c["fovy"],
                         step, RAMP, termination=term)
        torch.cuda.synchronize()
        f32 = lambda x: [float(np.float32(t)) for t in x]
        ref = oracle.render(v, 0.0, 1.0, 40, 30, f32(c["eye"]), f32(c["center"]), f32(c["up"]),
                            float(np.float32(c["fovy"])), float(np.float32(step)),
                            float(np.float32(term)), (0, 0, 0, 0), RAMP)
        err = np.max(np.abs(got.cpu().numpy().astype(np.float64) - ref))
        assert err <= TOL, f"step {step} termination {term}: {err:.2e}"


def test_render_rejects_bad_parameters():
    v = torch.from_numpy(volume(synth.U8, (8, 8, 8), SEED)).cuda()
    with pytest.raises(vkt.VktError):
        vkt.render(v, 8, 8, (4, 4, -10), (4, 4, 4), (0, 0, 1), 0.8, 0.5, RAMP)   # up parallel to view
    with pytest.raises(vkt.VktError):
        vkt.render(v, 8, 8, (4, 4, -10), (4, 4, 4), (0, 1, 0), 0.8, 0.0, RAMP)   # zero step
    with pytest.raises(vkt.VktError):
        vkt.render(v, 8, 8, (4, 4, -10), (4, 4, 4), (0, 1, 0), 0.8, 0.5, RAMP[:1])  # one entry


def test_render_full_size_sampled():
    """The bench's frame: 1024 x 768 of the 512^3 uint8 CT-like volume, step 0.5, the ramp
    table; 2000 seeded pixels (and the four corners and the centre) against the oracle."""
    v = synth.volume("blobs", synth.U8, (512, 512, 512), synth.BASE_SEED + 1)
    W, H = 1024, 768
    eye, center, up, fovy = (256.0, 300.0, -600.0), (256.0, 256.0, 256.0), (0.0, 1.0, 0.0), 0.8
    lut = np.array([[0, 0, 0, 0], [0.9, 0.5, 0.2, 0.02], [1, 0.9, 0.6, 0.15], [1, 1, 1, 0.6]], np.float32)
    img = vkt.render(torch.from_numpy(v).cuda(), W, H, eye, center, up, fovy, 0.5, lut)
    torch.cuda.synchronize()
    rng = np.random.default_rng(SEED + 55)
    pix = np.concatenate([np.array([[0, 0], [W - 1, 0], [0, H - 1], [W - 1, H - 1], [W // 2, H // 2]]),
                          np.stack([rng.integers(0, W, 2000), rng.integers(0, H, 2000)], axis=1)])
    f32 = lambda x: [float(np.float32(t)) for t in x]
    ref = oracle.render_pixels(v, 0.0, 1.0, W, H, f32(eye), f32(center), f32(up),
                               float(np.float32(fovy)), 0.5, 2.0, (0, 0, 0, 0), lut, pix)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]].astype(np.float64)
    err = np.max(np.abs(got - ref))
    assert err <= TOL, f"max |gpu - oracle| = {err:.2e}"
