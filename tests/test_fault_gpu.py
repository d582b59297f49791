"""Failure detection on the GPU without a fault: a withheld TMA load makes one bounded wait
run out, the kernel reports the timeout through the device status word, and the context
stays usable for the next call (which must again agree with the oracle).

The injection is the policy flag VKT_DEBUG_INJECT_WAIT_TIMEOUT: each CTA of the direct path
skips the load of its first input plane, so no trap, bad address or unbounded loop is
involved; every wait in the kernel gives up after 2 s.
"""
import re
import time
from pathlib import Path

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

import paper_2203_10213_gb300 as vkt  # noqa: E402
from gpu_util import compare  # noqa: E402

HEADER = Path(__file__).resolve().parents[1] / "include" / "vkt.h"


def test_debug_flags_match_header():
    defs = dict(re.findall(r"#define (VKT_DEBUG_\w+) (\d+)", HEADER.read_text()))
    assert int(defs["VKT_DEBUG_LOG"]) == vkt.DEBUG_LOG
    assert int(defs["VKT_DEBUG_INJECT_WAIT_TIMEOUT"]) == vkt.DEBUG_INJECT_WAIT_TIMEOUT


@pytest.mark.gpu
def test_injected_wait_timeout_is_reported_and_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # 48 x 32 x 24 uint8 (rows of 48 bytes: tensor-map capable), dense Laplacian, direct path
    vol = synth.volume("blobs", synth.U8, (48, 32, 24), synth.BASE_SEED + 41)
    assert vol.shape == (24, 32, 48)
    w = synth.laplacian_3()
    filt = vkt.Filter.dense(w)
    src = torch.from_numpy(vol).cuda()
    out = torch.full(vol.shape, -7.0, dtype=torch.float32, device="cuda")
    vkt.synchronize()

    with vkt.policy(path="direct", debug=vkt.DEBUG_INJECT_WAIT_TIMEOUT):
        vkt.filter_tensor(src, filt, out=out)
        t0 = time.monotonic()
        code = vkt._lib.vktSynchronize()
        waited = time.monotonic() - t0
    assert vkt.ERRORS.get(code) == "VKT_ERROR_DEVICE_TIMEOUT", code
    assert waited > 1.0, f"the bounded wait returned after {waited:.2f} s"
    # the CTAs exited without writing
    assert bool((out == -7.0).all())
    # the status was cleared and the context is usable
    assert vkt._lib.vktSynchronize() == 0
    vkt.filter_tensor(src, filt, out=out, path="direct")
    vkt.synchronize()
    ref = oracle.correlate(vol, w, 0.0, 1.0)
    compare(out.cpu().numpy(), ref, w, vol, (0.0, 1.0), (0.0, 1.0), "after injected timeout")
