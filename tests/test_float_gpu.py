"""GPU parity of the float32 variant and its hand-written adjoint against the
FP64 oracle (max abs error 1e-4), through the C ABI and through autograd."""
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


def test_full_size_batch_sampled(codec):
    """64 x 3 x 512 x 512 float32 N(0,1): whole batch on the GPU, sampled planes vs FP64."""
    shape = (64, 3, 512, 512)
    x = inputs.normal_batch(shape, seed=inputs.BASE_SEED)
    xd = torch.from_numpy(x).to(DEV)
    Q = np.ones(64)
    y = codec.forward_f32(xd, Q)
    gx = codec.backward_f32(xd, y, Q)
    torch.cuda.synchronize()
    for (b, c) in ((0, 0), (31, 2), (63, 1)):
        xp = x[b, c][None].astype(np.float64)
        yp = oracle.forward_f64(xp, Q)
        assert np.abs(y[b, c].cpu().numpy() - yp[0]).max() <= TOL
        assert np.abs(gx[b, c].cpu().numpy() - oracle.backward_f64(xp, yp, Q)[0]).max() <= 2 * TOL


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
