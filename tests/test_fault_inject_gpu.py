"""Failure paths, injected on the host (no GPU fault): ADCT_FAULT_INJECT=alloc:K
makes the K-th device allocation of the process fail as if the device were
out of memory.  Each case runs in a fresh process; the entry point that hit
the failure returns ADCT_ERR_OOM, and the same process then goes on to
produce correct results."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRELUDE = f"""
import sys
sys.path.insert(0, {ROOT!r})
import numpy as np, torch
import oracle
from paper_1702_00817_gb300 import _native, inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, AdctError, Codec, Image, make_quant
dev = torch.device("cuda:0")
img = inputs.synth_image(64, 96, 3)[0]
Q = inputs.step_table(4)
q = make_quant(ADCT_Q_STEP, Q)
def roundtrip(codec):
    src = torch.from_numpy(img).to(dev)
    dst = torch.empty_like(src)
    coef = torch.empty((1, 8, 12, 8, 8), dtype=torch.int16, device=dev)
    codec.roundtrip([Image(src, dst, coef)], q)
    torch.cuda.synchronize()
    qr, rr = oracle.roundtrip(img, oracle.MODE_STEP, Q, 64)
    assert np.array_equal(dst.cpu().numpy(), rr) and np.array_equal(coef[0].cpu().numpy().astype(np.int64), qr)
def expect_oom(fn):
    try:
        fn()
    except AdctError as e:
        assert e.status == _native.ADCT_ERR_OOM, e
        return
    raise AssertionError("no error")
"""


def _run(k: int, body: str):
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, ADCT_FAULT_INJECT=f"alloc:{k}")
    out = subprocess.run([sys.executable, "-c", PRELUDE + body + "\nprint('PASS')"], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0 and "PASS" in out.stdout, out.stdout + out.stderr


def test_context_creation_fails_cleanly_then_works():
    _run(1, "expect_oom(lambda: Codec(0))\nc = Codec(0)\nroundtrip(c)\nc.close()")


def test_workspace_allocation_fails_then_the_context_recovers():
    _run(2, "c = Codec(0)\nexpect_oom(lambda: roundtrip(c))\nroundtrip(c)\nroundtrip(c)\nc.close()")


def test_server_arena_allocation_fails_cleanly():
    _run(2, """
from paper_1702_00817_gb300.serve import NativeServer
expect_oom(lambda: NativeServer(0, budget_bytes=64 << 20, quant=q))
srv = NativeServer(0, budget_bytes=64 << 20, quant=q)
r = srv.encode(torch.from_numpy(img).pin_memory())
assert r.done.wait(30) and r.error is None
d = srv.decode(r.result)
assert d.done.wait(30) and d.error is None
assert np.array_equal(d.result.numpy(), oracle.roundtrip(img, oracle.MODE_STEP, Q, 64)[1])
srv.close()
""")
