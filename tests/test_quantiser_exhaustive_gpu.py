"""Exhaustive GPU check of the step quantiser with D^2 merged (Sec. 2) over
its whole input domain, against the oracle's exact rational rounding.

Coefficients of 8-bit pixels obey |Z_ij| <= 128 2^(a_i + a_j) <= 8192 (the
rows of T have L1 norms 2^a_i, Sec. 2), so Z in [-8192, 8192] is the
quantiser's whole input domain, and a step is any uint16 Q >= 1.  The kernel
divides with a multiply-high by ceil(2^32 / Q), corrects ties for even steps
with a byte permute, and short-cuts Q > 16384 to zero; none of that is in the
oracle, which rounds the exact fraction.  Both sides compute integers, so the
comparison is bit for bit.

Coefficient leg: every Z in [-8192, 8192] at every one of the 64 positions,
for every Q in [1, 16448] (64 consecutive steps per table, both parities:
the kernel with the tie correction), every odd Q in [1, 16511] (tables of odd
steps only: the kernel without it), Q in (16448, 65535] on a stride that
alternates parity, and the zonal step quantiser on some of those tables.

Pixel leg: the fused round trip folds the level shift into the constant of
position (0, 0).  Constant blocks c = 0..255 give Z_00 = 64 (c - 128) and
Z_ij = 0 elsewhere; every Q_00 in [1, 16448] (with odd steps elsewhere, so
the tie-correcting kernel runs exactly when Q_00 is even), every odd Q_00 in
that range again beside even steps (the tie-correcting kernel with an odd
Q_00), and Q_00 in (16448, 65535] on a stride; q and the reconstructed
pixels are compared with the oracle's round trip."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, ADCT_Q_STEP_ZONAL, Codec, Image, make_quant

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ZMAX = 8192
HB, WB = 145, 113  # 145 * 113 = 16385 blocks: one per Z in [-8192, 8192]
CHUNK = 32         # tables in flight per synchronisation
POOL = ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1)))


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    c = Codec(0)
    yield c
    c.close()


def _coef_tables():
    """(mode, Q table, r) of the coefficient leg."""
    out = []
    for t in range(257):  # every step 1..16448, consecutive
        out.append((ADCT_Q_STEP, np.arange(64 * t + 1, 64 * t + 65), 64))
    for t in range(129):  # every odd step 1..16511, odd-only tables
        out.append((ADCT_Q_STEP, 1 + 2 * (64 * t + np.arange(64)), 64))
    big = np.arange(16449, 65536, 13)  # 13 is odd: parities alternate
    big = np.concatenate([big, [65534, 65535]])
    big = np.concatenate([big, np.full((-big.size) % 64, 65535)])
    for t in range(big.size // 64):
        out.append((ADCT_Q_STEP, big[64 * t: 64 * t + 64], 64))
    for t, r in ((0, 1), (1, 21), (128, 37), (256, 64)):
        out.append((ADCT_Q_STEP_ZONAL, np.arange(64 * t + 1, 64 * t + 65), r))
    out.append((ADCT_Q_STEP_ZONAL, 1 + 2 * np.arange(64), 10))
    return [(m, q.astype(np.uint16), r) for m, q, r in out]


def test_quantiser_exhaustive_on_coefficients(codec):
    zvals = np.arange(-ZMAX, ZMAX + 1, dtype=np.int64)
    Z = np.repeat(zvals[:, None], 64, axis=1).reshape(HB, WB, 8, 8)
    template = torch.from_numpy(Z.astype(np.int16)[None]).to(DEV)
    tables = _coef_tables()
    work = torch.empty((CHUNK,) + tuple(template.shape), dtype=torch.int16, device=DEV)
    covered = np.zeros(65536, bool)

    def check(got, mode, Q, r):
        expect = oracle.quantise(Z, oracle.MODE_STEP if mode == ADCT_Q_STEP else oracle.MODE_STEP_ZONAL, Q, r)
        bad = np.argwhere(got.astype(np.int64) != expect)
        return None if bad.size == 0 else (mode, r, bad[0].tolist(), Q.reshape(8, 8)[tuple(bad[0][2:])])

    for c0 in range(0, len(tables), CHUNK):
        part = tables[c0: c0 + CHUNK]
        for k, (mode, Q, r) in enumerate(part):
            work[k].copy_(template)
            codec.quantise([Image(None, None, work[k])], make_quant(mode, Q, r))
        torch.cuda.synchronize()
        host = work[: len(part)].cpu().numpy()[:, 0]
        fails = [f for f in POOL.map(lambda a: check(host[a[0]], *a[1]), enumerate(part)) if f]
        assert not fails, fails[:3]
        for mode, Q, r in part:
            covered[Q] = True
    assert covered[1:16449].all() and covered[65535]


def _const_blocks_image():
    c = np.arange(256, dtype=np.uint8).reshape(16, 16)
    return np.repeat(np.repeat(c, 8, axis=0), 8, axis=1)  # block (by, bx) is constant 16 by + bx


def test_pixel_path_dc_constant_exhaustive(codec):
    img = _const_blocks_image()
    src = torch.from_numpy(img).to(DEV)
    odd_rest = (2 * np.add.outer(np.arange(8), np.arange(8)) + 1).reshape(64)  # odd steps off (0, 0)
    even_rest = inputs.step_table(1).reshape(64).astype(np.int64)             # 2 + i + j: even steps too
    runs = [(q00, odd_rest) for q00 in range(1, 16449)]
    runs += [(q00, even_rest) for q00 in range(1, 16449, 2)]
    runs += [(q00, odd_rest) for q00 in range(16449, 65536, 97)] + [(65535, odd_rest), (65534, even_rest)]
    batch = 512
    coef = torch.empty((batch, 16, 16, 8, 8), dtype=torch.int16, device=DEV)
    dst = torch.empty((batch, 128, 128), dtype=torch.uint8, device=DEV)

    def check(k, q00, rest, qh, dh):
        Q = rest.copy()
        Q[0] = q00
        q_ref, rec_ref = oracle.roundtrip(img, oracle.MODE_STEP, Q.astype(np.uint16))
        if not np.array_equal(qh.astype(np.int64), q_ref):
            return ("q", q00, int(rest[1]))
        if not np.array_equal(dh, rec_ref):
            return ("pixels", q00, int(rest[1]))
        return None

    for c0 in range(0, len(runs), batch):
        part = runs[c0: c0 + batch]
        for k, (q00, rest) in enumerate(part):
            Q = rest.copy()
            Q[0] = q00
            codec.roundtrip([Image(src, dst[k], coef[k][None])], make_quant(ADCT_Q_STEP, Q.astype(np.uint16)))
        torch.cuda.synchronize()
        qh = coef[: len(part)].cpu().numpy()
        dh = dst[: len(part)].cpu().numpy()
        fails = [f for f in POOL.map(lambda a: check(a[0], a[1][0], a[1][1], qh[a[0]], dh[a[0]]),
                                     enumerate(part)) if f]
        assert not fails, fails[:3]
