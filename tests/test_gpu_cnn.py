"""CUDA kernels of the elimination proposal network against the FP64
reference (oracle/cnn.py), evaluated with the BF16-rounded weights the kernels
use: probabilities, loss and the full parameter gradient; and Adam steps
through the C ABI lower the loss on a fixed batch."""
import numpy as np
import pytest

import oracle.cnn as ocnn
import oracle.learned as ol
import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_08606_gb300 import build, binding
    build()
    binding.load()
    return binding


def _batch(seed, Bn, H, W):
    s = scenegen.Stream(seed, 7)
    x = s.normal(Bn * 6 * H * W).reshape(Bn, 6, H, W).astype(np.float32)
    y = (s.uniform(Bn * H * W) < 0.25).astype(np.float32).reshape(Bn, H, W)
    return x, y


@pytest.mark.parametrize("Bn,H,W", [(1, 16, 16), (2, 19, 33), (3, 32, 32)])
def test_forward_and_gradient_match_fp64(B, Bn, H, W):
    dev = torch.device("cuda:0")
    net = B.CNN(H, W, max_batch=Bn)
    p = scenegen.cnn_init(11, scale=0.9, head_bias=-0.5)
    net.set_params(p)
    pr = ol.round_bf16(p)
    # the weights the kernels use are exactly the round-to-nearest-even BF16 values
    assert np.array_equal(net.params(rounded=True).astype(np.float64), pr)
    x, y = _batch(H + W, Bn, H, W)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    prob = net.forward(xt).cpu().numpy()
    ref, _ = ocnn.forward(pr, x.astype(np.float64))
    assert np.max(np.abs(prob - ref)) <= 2e-5
    g, loss = net.backward(xt, yt, pos_weight=3.0)
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = ocnn.loss_and_grad(pr, x.astype(np.float64), y.astype(np.float64), 3.0)
    assert abs(loss - lref) <= 1e-6 * max(1.0, abs(lref))
    o = 0
    for name, shape in ocnn.layout():
        n = int(np.prod(shape))
        gb, rb = g[o:o + n], gref[o:o + n]
        assert np.linalg.norm(gb - rb) <= 1e-4 * np.linalg.norm(rb) + 1e-9, name
        o += n
    net.close()


def test_adam_steps_lower_the_loss(B):
    dev = torch.device("cuda:0")
    H = W = 32
    net = B.CNN(H, W, max_batch=4)
    net.set_params(scenegen.cnn_init(3, head_bias=-1.0))
    x, y = _batch(5, 4, H, W)
    # a learnable target: pixels whose first feature exceeds 0.5
    y = (x[:, 0] > 0.5).astype(np.float32)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    _, l0 = net.backward(xt, yt)
    for _ in range(60):
        g, _ = net.backward(xt, yt)
        net.adam_step(g, 3e-3)
    _, l1 = net.backward(xt, yt)
    assert l1 < 0.5 * l0
    net.close()
