"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and its own butterfly (run on the host through the diagnostic entry
point) equals the oracle's dense T with exactly 14 additions (Table 1)."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from paper_1702_00817_gb300 import _build, _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _native.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "adct.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(_native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in [(0, "ADCT_OK"), (2, "ADCT_ERR_SHAPE"), (5, "ADCT_ERR_CUDA"), (7, "ADCT_ERR_UNSUPPORTED")]:
        assert lib.adct_status_string(code).decode() == name


def test_butterfly_equals_dense_T_on_all_ternary_vectors(lib):
    from paper_1702_00817_gb300.codec import butterfly_host
    T = oracle.matrix_T()
    vecs = np.array(list(itertools.product((-1, 0, 1), repeat=8)), np.int32)
    out, adds = butterfly_host(vecs)
    assert adds == 14
    assert np.array_equal(out.astype(np.int64), vecs.astype(np.int64) @ T.T)
    out_i, adds_i = butterfly_host(vecs, inverse=True)
    assert adds_i == 14
    assert np.array_equal(out_i.astype(np.int64), vecs.astype(np.int64) @ T)


def test_butterfly_on_unit_and_random_vectors(lib):
    from paper_1702_00817_gb300.codec import butterfly_host
    T = oracle.matrix_T()
    rng = np.random.default_rng(1)
    vecs = np.concatenate([np.eye(8, dtype=np.int32),
                           rng.integers(-255, 256, size=(100000, 8)).astype(np.int32)])
    out, adds = butterfly_host(vecs)
    assert adds == 14
    assert np.array_equal(out.astype(np.int64), vecs.astype(np.int64) @ T.T)
    # inverse after forward, with 64 D^2 applied between: T^T (64 D^2) T x = 64 x
    a = oracle.scale_exponents()
    back, _ = butterfly_host((out.astype(np.int64) * (64 >> a)).astype(np.int32), inverse=True)
    assert np.array_equal(back.astype(np.int64), 64 * vecs.astype(np.int64))


def test_create_without_device_fails_cleanly(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.adct_create(ctypes.byref(h), 0) != 0
    assert not h.value


def test_make_quant_validates():
    from paper_1702_00817_gb300.codec import make_quant
    q = make_quant(1, np.arange(1, 65), 10)
    assert q.mode == 1 and q.r == 10 and list(q.Q)[:3] == [1, 2, 3]
    with pytest.raises(ValueError):
        make_quant(1, np.arange(1, 10))
    with pytest.raises(ValueError):
        make_quant(1, np.full(64, 70000))


def test_shard_plan_is_a_balanced_partition():
    from paper_1702_00817_gb300 import _native, inputs
    from paper_1702_00817_gb300.codec import AdctError, shard_plan
    sizes = inputs.ragged_sizes(1000, seed=3)
    blocks = [(h // 8) * (w // 8) for h, w in sizes]
    for world in (1, 2, 3, 8):
        plans = [shard_plan(sizes, world, r) for r in range(world)]
        idx = sorted(i for p, _ in plans for i in p)
        assert idx == list(range(len(sizes)))                     # every image exactly once
        loads = [sum(blocks[i] for i in p) for p, _ in plans]
        assert all(mx == max(loads) for _, mx in plans)
        assert max(loads) <= sum(blocks) / world + max(blocks)    # list-scheduling bound
        assert all(p == sorted(p) for p, _ in plans)
    assert shard_plan(sizes, 1, 0)[0] == list(range(len(sizes)))
    # ties: equal images alternate over the ranks in index order
    assert shard_plan([(8, 8)] * 4, 2, 0)[0] == [0, 2]
    assert shard_plan([], 4, 3) == ([], 0)
    for bad in ((2, 2), (2, -1), (0, 0)):
        with pytest.raises(AdctError) as e:
            shard_plan(sizes, *bad)
        assert e.value.status == _native.ADCT_ERR_INVALID_ARG
    for bad_shape in ((0, 8), (8, 65544), (0, 8, 8)):
        with pytest.raises(AdctError) as e:
            shard_plan([bad_shape], 2, 0)
        assert e.value.status == _native.ADCT_ERR_SHAPE
    # any side: edge blocks count whole, ceil(side / 8) per side
    assert shard_plan([(12, 8), (9, 17)], 1, 0) == ([0, 1], 2 + 2 * 3)
    assert shard_plan([(1, 1)] * 3, 2, 1) == ([1], 2)


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """The header is plain C (C11, no CUDA headers needed) and a C program
    links against the library and calls it; without a GPU, context creation
    fails with a status, not a crash."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_adct.c"
    src.write_text('#include "adct.h"\n#include <stdio.h>\n'
                   "int main(void) {\n"
                   "  adct_context* ctx = NULL;\n"
                   "  adct_status st = adct_create(&ctx, 0);\n"
                   '  printf("%s\\n", adct_status_string(st));\n'
                   "  if (st == ADCT_OK) adct_destroy(ctx);\n"
                   "  return 0;\n}\n")
    libdir = os.path.dirname(_build.LIB)
    exe = tmp_path / "use_adct"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-ladct", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip().startswith("ADCT_")


def test_shard_plan_properties_on_random_batches():
    """Random batches (hypothesis): every rank's list is sorted, the lists
    partition the batch, the reported maximum is the largest rank load, and
    the load spread stays within the largest image (greedy list scheduling)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from paper_1702_00817_gb300.codec import shard_plan

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(st.lists(st.tuples(st.integers(1, 4), st.integers(1, 600), st.integers(1, 600)), max_size=40),
               st.integers(1, 9))
    def check(shapes, world):
        blocks = [c * ((h + 7) // 8) * ((w + 7) // 8) for c, h, w in shapes]
        plans = [shard_plan(shapes, world, r) for r in range(world)]
        assert sorted(i for p, _ in plans for i in p) == list(range(len(shapes)))
        loads = [sum(blocks[i] for i in p) for p, _ in plans]
        assert all(p == sorted(p) and mx == max(loads, default=0) for (p, mx) in plans)
        if blocks:
            assert max(loads) - min(loads) <= max(blocks)

    check()


def _fake_planar(channels, side=8):
    """An adct_image with aligned placeholder pointers; only validation reads it."""
    im = _native.adct_image()
    im.src, im.dst = 0x10000, 0x20000
    im.width = im.height = side
    im.channels = channels
    im.layout = _native.ADCT_LAYOUT_PLANAR
    im.pitch, im.plane_stride = side, side * side
    return im


def _noalloc_args(images):
    import ctypes
    from paper_1702_00817_gb300.codec import ADCT_Q_STEP, make_quant
    arr = (_native.adct_image * len(images))(*images)
    return arr, make_quant(ADCT_Q_STEP, np.full(64, 3))


def test_noalloc_plane_count_cannot_overflow(lib):
    # A channel count near INT32_MAX after other planes must be refused as too
    # large, not wrap the running plane count past the table's limit.  Checked
    # on the host before any device work, so no GPU is involved.
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("placeholder pointers: host-only check")
    for first, second in ((1, 2 ** 31 - 1), (1023, 2), (1000, 2 ** 31 - 1000)):
        arr, q = _noalloc_args([_fake_planar(first), _fake_planar(second)])
        assert lib.adct_roundtrip_noalloc(arr, 2, ctypes.byref(q), None) == _native.ADCT_ERR_TOO_LARGE


def test_noalloc_table_fits_a_small_thread_stack(lib):
    # The 72 KiB descriptor table is built in a library buffer, not on the
    # caller's stack: a full 1024-plane batch from a thread with a 64 KiB stack
    # gets through validation and table building to the device lookup (which
    # fails here, with no GPU) instead of overflowing the stack.
    import ctypes
    import threading
    import torch
    if torch.cuda.is_available():
        pytest.skip("placeholder pointers: host-only check")
    arr, q = _noalloc_args([_fake_planar(4) for _ in range(256)])
    out = []
    old = None
    for size in (65536, 131072):  # 128 KiB where that is the platform's minimum (aarch64, 64 KiB pages)
        try:
            old = threading.stack_size(size)
            break
        except ValueError:
            continue
    assert old is not None
    try:
        t = threading.Thread(target=lambda: out.append(lib.adct_roundtrip_noalloc(arr, 256, ctypes.byref(q), None)))
        t.start()
        t.join()
    finally:
        threading.stack_size(old)
    assert out == [_native.ADCT_ERR_CUDA]
