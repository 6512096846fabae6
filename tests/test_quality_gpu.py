"""Quality measures of the image experiment (Sec. 3): the per-plane squared
error of the round trip (exact against the oracle) and of the exact-DCT
comparator (float32 against the FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, ADCT_Q_ZONAL, Codec, Image, make_quant

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    c = Codec(0)
    yield c
    c.close()


def _planes(imgs):
    return [x[c] for x in imgs for c in range(x.shape[0])]


@pytest.mark.parametrize("mode,Q,r", [(ADCT_Q_ZONAL, None, 1), (ADCT_Q_ZONAL, None, 10), (ADCT_Q_ZONAL, None, 45),
                                      (ADCT_Q_ZONAL, None, 64), (ADCT_Q_STEP, 1, 64), (ADCT_Q_STEP, 16, 64)])
def test_roundtrip_sse_is_exact(codec, mode, Q, r):
    sizes = inputs.ragged_sizes(5, seed=31, lo_log2=4.0, hi_log2=8.0)
    imgs = inputs.ragged_batch(sizes, channels=2, base_seed=31)
    Qt = inputs.step_table(Q) if Q else None
    srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
    got = codec.quality([Image(s) for s in srcs], make_quant(mode, Qt, r)).cpu().numpy()
    omode = oracle.MODE_ZONAL if mode == ADCT_Q_ZONAL else oracle.MODE_STEP
    want = [oracle.sse(oracle.roundtrip(p, omode, Qt, r)[1], p) for p in _planes(imgs)]
    assert got.tolist() == want
    if mode == ADCT_Q_ZONAL and r == 64:
        assert not got.any()


@pytest.mark.parametrize("r", [1, 6, 25, 45, 64])
def test_dct_comparator_matches_fp64(codec, r):
    imgs = [inputs.synth_image(96, 128, 40 + k) for k in range(3)]
    srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
    got = codec.quality_dct([Image(s) for s in srcs], r).cpu().numpy()
    want = np.array([oracle.sse(oracle.dct_zonal(p, r), p) for p in _planes(imgs)])
    # float32 against float64: a reconstruction that lands on a rounding tie can
    # differ by one grey level, so allow a relative 1e-3 (and exact zero at r = 64)
    assert np.all(np.abs(got - want) <= 1e-3 * np.maximum(want, 1) + 2)
    if r == 64:
        assert not got.any()
