"""The ragged batch at full size (1000 three-channel images, sides log-uniform
over 64..4096, 44 M blocks) in the benchmark's form -- autotuned, one
graph-captured launch -- checked against the oracle on every plane, bit for
bit (the oracle runs on the host cores in threads)."""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, Codec, Image, make_quant

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_full_ragged_batch_every_plane_against_the_oracle():
    import __graft_entry__
    __graft_entry__.build()
    n = 1000
    sizes = inputs.ragged_sizes(n, seed=inputs.BASE_SEED)
    srcs = [inputs.synth_image_device(h, w, inputs.BASE_SEED + i, 3, DEV) for i, (h, w) in enumerate(sizes)]
    dsts = [torch.empty_like(x) for x in srcs]
    coefs = [torch.empty((3, h // 8, w // 8, 8, 8), dtype=torch.int16, device=DEV) for h, w in sizes]
    images = [Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)]
    Q = inputs.step_table(4)
    q = make_quant(ADCT_Q_STEP, Q)
    with Codec(0) as codec:
        codec.autotune(images, q, reps=1)
        for d in dsts:
            d.fill_(0)
        codec.roundtrip_graph(images, q)
        codec.roundtrip_graph(images, q)  # a replay
        torch.cuda.synchronize()

    def check(i):
        x, d, c = srcs[i].cpu().numpy(), dsts[i].cpu().numpy(), coefs[i].cpu().numpy()
        for k in range(3):
            q_ref, rec_ref = oracle.roundtrip(x[k], oracle.MODE_STEP, Q, 64)
            if not (np.array_equal(c[k].astype(np.int64), q_ref) and np.array_equal(d[k], rec_ref)):
                return i
        return None

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        bad = [i for i in ex.map(check, range(n)) if i is not None]
    assert bad == [], f"images differing from the oracle: {bad[:10]}"
