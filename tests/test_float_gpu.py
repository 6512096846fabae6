"""GPU parity of the float32 variant and its hand-written adjoint against the
FP64 oracle (max abs error 1e-4), through the C ABI and through autograd."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.autograd import ADCTFunction, default_codec

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-4
QS = {"none": None, "ones": np.ones(64), "step1": inputs.step_table(1).astype(np.float64),
      "half": np.full(64, 0.5)}


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    return default_codec(0)


@pytest.mark.parametrize("qname", list(QS))
@pytest.mark.parametrize("shape", [(1, 8, 8), (3, 64, 64), (2, 40, 136), (5, 8, 264)])
def test_forward_backward_match_fp64(codec, qname, shape):
    Q = QS[qname]
    x = inputs.normal_batch(shape, seed=sum(shape))
    g = inputs.normal_batch(shape, seed=sum(shape) + 1)
    xd, gd = torch.from_numpy(x).to(DEV), torch.from_numpy(g).to(DEV)
    y = codec.forward_f32(xd, Q)
    gx = codec.backward_f32(xd, gd, Q)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - oracle.forward_f64(x, Q)).max() <= TOL
    assert np.abs(gx.cpu().numpy() - oracle.backward_f64(x, g, Q)).max() <= TOL


def test_autograd_function(codec):
    Q = inputs.step_table(1).astype(np.float64)
    x = inputs.normal_batch((2, 3, 32, 48), seed=4)
    g = inputs.normal_batch(x.shape, seed=5)
    xd = torch.from_numpy(x).to(DEV).requires_grad_(True)
    y = ADCTFunction.apply(xd, Q)
    (y * torch.from_numpy(g).to(DEV)).sum().backward()
    torch.cuda.synchronize()
    assert np.abs(y.detach().cpu().numpy() - oracle.forward_f64(x, Q)).max() <= TOL
    assert np.abs(xd.grad.cpu().numpy() - oracle.backward_f64(x, g, Q)).max() <= TOL


@pytest.mark.parametrize("qname", ["ones", "step1"])
def test_full_size_batch_every_plane(codec, qname):
    """64 x 3 x 512 x 512 float32 N(0,1), the whole batch in one launch each
    way, every one of the 192 planes against FP64 (oracle in threads), forward
    and adjoint both held to 1e-4."""
    shape = (64, 3, 512, 512)
    Q = QS[qname]
    x = inputs.normal_batch(shape, seed=inputs.BASE_SEED)
    g = inputs.normal_batch(shape, seed=inputs.BASE_SEED + 1)
    xd, gd = torch.from_numpy(x).to(DEV), torch.from_numpy(g).to(DEV)
    y = codec.forward_f32(xd, Q)
    gx = codec.backward_f32(xd, gd, Q)
    torch.cuda.synchronize()
    yh, gxh = y.cpu().numpy().reshape(-1, 512, 512), gx.cpu().numpy().reshape(-1, 512, 512)
    xh, gh = x.reshape(-1, 512, 512), g.reshape(-1, 512, 512)
    del xd, gd, y, gx

    def err(p):
        xp = xh[p][None].astype(np.float64)
        ey = np.abs(yh[p] - oracle.forward_f64(xp, Q)[0]).max()
        eg = np.abs(gxh[p] - oracle.backward_f64(xp, gh[p][None], Q)[0]).max()
        return ey, eg

    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as pool:
        errs = np.array(list(pool.map(err, range(xh.shape[0]))))
    assert errs[:, 0].max() <= TOL, errs[:, 0].max()
    assert errs[:, 1].max() <= TOL, errs[:, 1].max()


@pytest.mark.parametrize("Qv", [0.5, 1.0, 3.0])
def test_soft_phase_over_many_periods(codec, Qv):
    """The kernels' own sin and cos of the soft quantiser's phase 2 pi y / Q
    (range reduction and truncated series) against FP64 on single-coefficient
    blocks whose coefficient y sweeps [-8, 8] (many periods, both signs; N(0,1)
    data stays inside) at 8 positions; held to 1e-5, ten times tighter than the
    path's tolerance, forward and adjoint."""
    d = 1.0 / np.sqrt(np.array([8, 2, 4, 2, 8, 2, 4, 2], np.float64))
    T = oracle.matrix_T().astype(np.float64)
    C = d[:, None] * T
    nblk = 4096
    amp = np.linspace(-8.0, 8.0, nblk)
    amp[:9] = Qv * np.array([-1, -0.75, -0.5, -0.25, 0, 0.25, 0.5, 0.75, 1])  # period landmarks
    Q = np.full(64, Qv)
    for (i, j) in ((0, 0), (0, 1), (1, 0), (2, 5), (3, 3), (7, 4), (6, 2), (7, 7)):
        basis = np.outer(C[i], C[j])
        x = np.concatenate([a * basis for a in amp], axis=1)[None].astype(np.float32)  # [1, 8, 8 nblk]
        gz = np.zeros_like(x)
        gz[0, i, j::8] = 1.0
        xd, gd = torch.from_numpy(x).to(DEV), torch.from_numpy(gz).to(DEV)
        y = codec.forward_f32(xd, Q)
        gx = codec.backward_f32(xd, gd, Q)
        torch.cuda.synchronize()
        x64 = x.astype(np.float64)
        assert np.abs(y.cpu().numpy() - oracle.forward_f64(x64, Q)).max() <= 1e-5, (i, j)
        assert np.abs(gx.cpu().numpy() - oracle.backward_f64(x64, gz.astype(np.float64), Q)).max() <= 1e-5, (i, j)


def test_float_argument_errors(codec):
    from paper_1702_00817_gb300.codec import AdctError
    x = torch.zeros((1, 12, 16), device=DEV)
    with pytest.raises(AdctError):
        codec.forward_f32(x)
    with pytest.raises(AdctError):
        codec.forward_f32(torch.zeros((1, 8, 8), device=DEV), np.zeros(64))


def test_float_binding_refuses_mismatched_or_host_tensors(codec):
    x = torch.zeros((2, 8, 16), device=DEV)
    with pytest.raises(ValueError):
        codec.backward_f32(x, torch.zeros((1, 8, 16), device=DEV))  # gy smaller than x
    with pytest.raises(ValueError):
        codec.forward_f32(x, out=torch.zeros((1, 8, 16), device=DEV))
    with pytest.raises(ValueError):
        codec.forward_f32(torch.zeros((2, 8, 16)))  # host tensor
