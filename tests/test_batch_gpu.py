"""GPU parity of the batched persistent launch (vktApplyFilterBatchSV) against the FP64
oracle, its CUDA-graph replay, and its agreement with one vktApplyFilterSV per volume."""
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

SEED = synth.BASE_SEED + 4
DT = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}


def make_batch(items, mixed_filters=False):
    out = []
    for j, it in enumerate(items):
        nx, ny, nz = it["dims"]
        fmt = it["fmt"]
        if fmt == synth.F32:
            src = synth.fourier(it["seed"], (nx, ny, nz), nmodes=8)
        else:
            src = synth.quantize(synth.blobs(it["seed"], (nx, ny, nz), nblobs=4,
                                             sigma=(2.0, 16.0)), fmt)
        k, sigma = it["k"], float(np.float32(it["sigma"]))
        if mixed_filters and j % 11 == 5:
            w = synth.normal(it["seed"] + 1, (k, k, k)).astype(np.float32)
            f = vkt.Filter.dense(w)
            wd = w.astype(np.float64)
        else:
            f = vkt.Filter.gaussian(k, sigma)
            wd = oracle.gaussian_weights(k, sigma)
        out.append(dict(src=src, fmt=fmt, filt=f, w=wd))
    return out


def run_batch(batch, reps=1):
    srcs, dsts, views_s, views_d = [], [], [], []
    for b in batch:
        s = torch.from_numpy(b["src"]).cuda()
        d = torch.empty(b["src"].shape, dtype=DT[b["fmt"]], device="cuda")
        srcs.append(s)
        dsts.append(d)
        views_s.append(vkt.StructuredVolume.from_tensor(s))
        views_d.append(vkt.StructuredVolume.from_tensor(d))
    for _ in range(reps):
        vkt.apply_filter_batch(views_d, views_s, [b["filt"] for b in batch])
    torch.cuda.synchronize()
    vkt.synchronize()
    return [d.cpu().numpy() for d in dsts]


def test_batch_mixed_small_matches_oracle():
    items = synth.batch_recipe(SEED, n=40, dmin=5, dmax=70)
    items[3]["k"], items[3]["sigma"] = 9, 3.0      # separable k=9: a single launch in the graph
    batch = make_batch(items, mixed_filters=True)
    outs = run_batch(batch)
    for j, (b, g) in enumerate(zip(batch, outs)):
        ref = oracle.correlate(b["src"], b["w"], 0.0, 1.0)
        compare(g, ref, b["w"], b["src"], (0, 1), (0, 1), f"batch item {j} fmt {b['fmt']}")


def test_batch_equals_single_launches():
    items = synth.batch_recipe(SEED + 1, n=24, dmin=8, dmax=96)
    batch = make_batch(items)
    outs = run_batch(batch, reps=2)               # the second call replays the cached graph
    for b, g in zip(batch, outs):
        s = torch.from_numpy(b["src"]).cuda()
        single = vkt.filter_tensor(s, b["filt"], dst_dtype=DT[b["fmt"]])
        torch.cuda.synchronize()
        assert np.array_equal(single.cpu().numpy(), g)


def test_batch_replay_picks_up_new_weights():
    items = synth.batch_recipe(SEED + 2, n=10, dmin=16, dmax=64)
    batch = make_batch(items)
    srcs = [torch.from_numpy(b["src"]).cuda() for b in batch]
    views_s = [vkt.StructuredVolume.from_tensor(s) for s in srcs]
    dsts = [torch.empty(b["src"].shape, dtype=torch.float32, device="cuda") for b in batch]
    views_d = [vkt.StructuredVolume.from_tensor(d) for d in dsts]
    vkt.apply_filter_batch(views_d, views_s, [b["filt"] for b in batch])
    # same handles, new Gaussian widths: the graph is replayed with the refreshed table
    filts2 = [vkt.Filter.gaussian(b["filt"].k, 0.7) for b in batch]
    vkt.apply_filter_batch(views_d, views_s, filts2)
    torch.cuda.synchronize()
    vkt.synchronize()
    for b, d, f in zip(batch, dsts, filts2):
        w = oracle.gaussian_weights(f.k, float(np.float32(0.7)))
        ref = oracle.correlate(b["src"], w, 0.0, 1.0)
        compare(d.cpu().numpy(), ref, w, b["src"], (0, 1), (0, 1), "replay")


def test_batch_full_config_sampled():
    """256 volumes, dims log-uniform in 16..256 per axis, u8/u16/f32 with the CT-like and
    turbulence-like value models, Gaussian k in {3,5,7} with sigma = k/3, dst = src format."""
    items = synth.batch_recipe(SEED + 3, n=256)
    batch = []
    for it in items:
        src = synth.volume(it["kind"], it["fmt"], it["dims"], it["seed"])
        sigma = float(np.float32(it["sigma"]))
        batch.append(dict(src=src, fmt=it["fmt"], filt=vkt.Filter.gaussian(it["k"], sigma),
                          w=oracle.gaussian_weights(it["k"], sigma)))
    outs = run_batch(batch)
    rng = np.random.default_rng(3)
    for j, (b, g) in enumerate(zip(batch, outs)):
        n = b["src"].size
        idx = np.unique(np.concatenate([rng.integers(0, n, 400), [0, n - 1]]))
        ref = oracle.correlate_points(b["src"], b["w"], idx, 0.0, 1.0)
        compare(g.ravel()[idx], ref, b["w"], b["src"], (0, 1), (0, 1), f"config item {j}")


def test_batch_rejects_bad_triples():
    a = torch.zeros((8, 8, 8), device="cuda")
    b = torch.zeros((8, 8, 9), device="cuda")
    va, vb = vkt.StructuredVolume.from_tensor(a), vkt.StructuredVolume.from_tensor(b)
    f = vkt.Filter.gaussian(3, 1.0)
    with pytest.raises(vkt.VktError):
        vkt.apply_filter_batch([va], [vb], [f])
    with pytest.raises(vkt.VktError):
        vkt.apply_filter_batch([va], [va], [f])          # in place
