"""The autotuner on the GPU: tuned calls (path and brick z extent chosen by timing) still
match the FP64 oracle, a tuned choice is recorded once per call shape and written to the
VKT_AUTOTUNE_CACHE file, a choice read from a file is the one used, batches are tuned per
plan, and nothing is timed while a stream is being captured."""
import ctypes
import json
import re

import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

SEED = synth.BASE_SEED + 11
lib = vkt._lib


def count():
    n = ctypes.c_int32()
    vkt.check(lib.vktAutotuneGetCount(ctypes.byref(n)))
    return n.value


@pytest.fixture
def fresh_tuner(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("VKT_AUTOTUNE_CACHE", str(path))
    vkt.check(lib.vktAutotuneSetEnabled(1))
    vkt.check(lib.vktAutotuneClear())
    yield path
    vkt.check(lib.vktAutotuneClear())


def entries(path):
    return {e["key"]: e for e in json.load(open(path))["entries"]}


@pytest.mark.parametrize("k", [5, 7])
def test_tuned_dense_call_matches_oracle_and_is_recorded(fresh_tuner, k):
    shape = (40, 48, 64)
    src = synth.uniform(SEED + k, shape, -1.0, 1.0)
    w = synth.normal(SEED + 10 + k, (k, k, k)).astype(np.float32)
    f = vkt.Filter.dense(w)
    gpu = run_gpu(vkt, src, f, torch.float32)          # first call: times the candidates
    assert count() == 1
    e = entries(fresh_tuner)
    (key, choice), = e.items()
    assert key.startswith(f"filter k{k} dense-tc s2 d2 volume 64x64x64"), key
    assert choice["path"] in (1, 3) and choice["ms"] > 0
    ref = oracle.correlate(src, w.astype(np.float64))
    compare(gpu, ref, w, src, (0, 1), (0, 1), f"tuned k={k}")
    gpu2 = run_gpu(vkt, src, f, torch.float32)         # second call: the recorded choice
    assert count() == 1
    assert np.array_equal(gpu, gpu2)


def test_choice_from_file_is_used(fresh_tuner, capfd):
    shape = (37, 70, 144)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = f"filter k3 separable s0 d2 volume 256x128x64 sm{sms}"
    fresh_tuner.write_text('{"vkt_autotune": 1, "entries": [\n'
                           + json.dumps({"key": key, "path": 2, "zchunk": 5, "ms": 1.0}) + "\n]}\n")
    vkt.check(lib.vktAutotuneClear())
    vkt.check(lib.vktAutotuneLoad(str(fresh_tuner).encode()))
    src = synth.quantize(synth.uniform(SEED + 20, shape), synth.U8)
    with vkt.policy(debug=vkt.DEBUG_LOG):
        gpu = run_gpu(vkt, src, vkt.Filter.gaussian(3, 1.0), torch.float32)
    log = capfd.readouterr().err
    assert re.search(r"\[vkt\] separable k=3 grid=\(\d+,\d+,8\) zchunk=5 ", log), log
    assert "autotune" not in log
    w = oracle.gaussian_weights(3, 1.0)
    compare(gpu, oracle.correlate(src, w, 0.0, 1.0), w, src, (0, 1), (0, 1), "file choice")


def test_tuned_batch_matches_oracle(fresh_tuner):
    items = synth.batch_recipe(SEED + 30, n=20, dmin=8, dmax=80)
    srcs, dsts, vs, vd, fs, ws = [], [], [], [], [], []
    dt = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}
    for it in items:
        a = synth.volume(it["kind"], it["fmt"], it["dims"], it["seed"])
        s = torch.from_numpy(a).cuda()
        d = torch.empty(a.shape, dtype=dt[it["fmt"]], device="cuda")
        sigma = float(np.float32(it["sigma"]))
        srcs.append(a)
        dsts.append(d)
        vs.append(vkt.StructuredVolume.from_tensor(s))
        vd.append(vkt.StructuredVolume.from_tensor(d))
        fs.append(vkt.Filter.gaussian(it["k"], sigma))
        ws.append(oracle.gaussian_weights(it["k"], sigma))
    vkt.apply_filter_batch(vd, vs, fs)
    torch.cuda.synchronize()
    vkt.synchronize()
    keys = [k for k in entries(fresh_tuner) if k.startswith("batch n20 ")]
    assert len(keys) == 1
    for a, d, w in zip(srcs, dsts, ws):
        compare(d.cpu().numpy(), oracle.correlate(a, w, 0.0, 1.0), w, a, (0, 1), (0, 1), "tuned batch")


def test_disabled_tuner_records_nothing(fresh_tuner):
    vkt.check(lib.vktAutotuneSetEnabled(0))
    try:
        src = synth.uniform(SEED + 40, (20, 24, 32), -1.0, 1.0)
        w = synth.normal(SEED + 41, (5, 5, 5)).astype(np.float32)
        gpu = run_gpu(vkt, src, vkt.Filter.dense(w), torch.float32)
        assert count() == 0
        compare(gpu, oracle.correlate(src, w.astype(np.float64)), w, src, (0, 1), (0, 1), "rule")
    finally:
        vkt.check(lib.vktAutotuneSetEnabled(1))


def test_no_timing_during_stream_capture(fresh_tuner):
    src = torch.from_numpy(synth.uniform(SEED + 50, (24, 40, 64), -1.0, 1.0)).cuda()
    w = synth.normal(SEED + 51, (3, 3, 3)).astype(np.float32)
    f = vkt.Filter.dense(w)
    out = torch.empty_like(src)
    vs, vo = vkt.StructuredVolume.from_tensor(src), vkt.StructuredVolume.from_tensor(out)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vkt.apply_filter(vo, vs, f, stream=s)
    assert count() == 0                 # the captured call used the rule, nothing was timed
    g.replay()
    torch.cuda.synchronize()
    ref = oracle.correlate(src.cpu().numpy(), w.astype(np.float64))
    compare(out.cpu().numpy(), ref, w, src.cpu().numpy(), (0, 1), (0, 1), "captured")
