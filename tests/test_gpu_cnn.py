"""The learned-guess network's GPU kernels (im2col + tcgen05 GEMM forward,
input and weight gradients, Adam) against the FP64 reference.  BF16
operands with FP32 accumulation: outputs within 3e-2 and gradients within
5e-2 relative (L2), set by BF16's 2^-9 rounding through four layers."""
import numpy as np
import pytest

from oracle import cnn_oracle as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_17634_gb300 import build
    build.build()
    from paper_2511_17634_gb300 import kp as K
    return K


def _init(ch, rng):
    layers = []
    for ci, co in zip(ch[:-1], ch[1:]):
        layers.append((rng.normal(scale=np.sqrt(2.0 / (9 * ci)), size=(co, ci, 3, 3)),
                       rng.normal(scale=0.05, size=co)))
    return R.flatten(layers)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_tap_orientation_exact(kp):
    ctx = kp.Context(max_n=4096)
    H, W = 7, 5
    net = kp.CNN(ctx, H, W, channels=(1, 1), max_batch=1)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 2, 0] = 1.0                       # di = +1, dj = -1: x[i+1, j-1]
    net.set_params(np.concatenate([w.ravel(), [0.0]]))
    x = np.arange(W * H, dtype=np.float64).reshape(1, 1, W, H) % 17
    xin = torch.as_tensor(x.reshape(1, 1, -1), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 1, W * H), dtype=torch.float32, device="cuda")
    net.forward(xin, out)
    torch.cuda.synchronize()
    ref = R.conv(x, w, np.zeros(1))
    assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref)


@pytest.mark.parametrize("H,W,B", [(16, 16, 2), (28, 20, 3)])
def test_forward_and_gradients_match_reference(kp, H, W, B):
    rng = np.random.default_rng(H * W + B)
    ch = (6, 32, 32, 32, 1)
    p = _init(ch, rng)
    x = rng.uniform(0, 1, size=(B, 6, W, H))
    t = rng.normal(scale=0.2, size=(B, 1, W, H))
    ctx = kp.Context(max_n=4096)
    net = kp.CNN(ctx, H, W, channels=ch, max_batch=B)
    net.set_params(p)
    xin = torch.as_tensor(x.reshape(B, 6, -1), dtype=torch.float32, device="cuda")
    tg = torch.as_tensor(t.reshape(B, 1, -1), dtype=torch.float32, device="cuda")
    out = torch.zeros((B, 1, H * W), dtype=torch.float32, device="cuda")
    net.forward(xin, out)
    grads = torch.zeros(net.nparams, dtype=torch.float32, device="cuda")
    loss = net.gradients(xin, tg, grads)
    torch.cuda.synchronize()
    ref_out = R.forward(p, ch, x)[-1]
    assert _rel(out.cpu().numpy().reshape(ref_out.shape), ref_out) <= 3e-2
    ref_loss, ref_g = R.loss_and_grads(p, ch, x, t)
    assert abs(loss - ref_loss) <= 3e-2 * ref_loss
    g = grads.cpu().numpy().astype(np.float64)
    o = 0
    for ci, co in zip(ch[:-1], ch[1:]):
        nw = co * ci * 9
        gw, rw = g[o:o + nw], ref_g[o:o + nw]
        gb, rb = g[o + nw:o + nw + co], ref_g[o + nw:o + nw + co]
        assert _rel(gw, rw) <= 5e-2, ("weights", ci, co, _rel(gw, rw))
        assert _rel(gb, rb) <= 5e-2, ("bias", ci, co, _rel(gb, rb))
        o += nw + co


def test_training_reduces_loss(kp):
    rng = np.random.default_rng(9)
    H, W, B = 16, 16, 4
    ch = (6, 32, 32, 32, 1)
    x = rng.uniform(0, 1, size=(B, 6, W, H))
    t = 0.5 * x[:, :1] - 0.3 * x[:, 1:2]          # a learnable target
    ctx = kp.Context(max_n=4096)
    net = kp.CNN(ctx, H, W, channels=ch, max_batch=B)
    net.set_params(_init(ch, rng))
    xin = torch.as_tensor(x.reshape(B, 6, -1), dtype=torch.float32, device="cuda")
    tg = torch.as_tensor(t.reshape(B, 1, -1), dtype=torch.float32, device="cuda")
    losses = [net.train_step(xin, tg, k + 1, lr=2e-3) for k in range(150)]
    assert losses[-1] < 0.05 * losses[0], (losses[0], losses[-1])


@pytest.mark.parametrize("H,W,B", [(7, 5, 1), (40, 30, 3), (128, 128, 10)])
def test_implicit_gemm_forward_exact_shifts(kp, H, W, B):
    # two one-tap layers shift the image twice; small integers keep every
    # product and sum exact in BF16 x BF16 -> FP32, so the tensor-core
    # implicit-GEMM path (padded-column layout, halo rows, several 512-row
    # super tiles per CTA at 128x128 x 10) must equal the FP64 reference bit
    # for bit, for every pair of taps
    rng = np.random.default_rng(H + W + B)
    x = rng.integers(0, 4, size=(B, 1, W, H)).astype(np.float64)
    xin = torch.as_tensor(x.reshape(B, 1, -1), dtype=torch.float32, device="cuda")
    out = torch.zeros((B, 1, W * H), dtype=torch.float32, device="cuda")
    ctx = kp.Context(max_n=16384)
    net = kp.CNN(ctx, H, W, channels=(1, 1, 1), max_batch=B)
    pairs = [(t1, t2) for t1 in range(9) for t2 in range(9)]
    if H * W > 4096:
        pairs = [(0, 8), (8, 0), (1, 7), (5, 3), (4, 4), (2, 6)]
    for t1, t2 in pairs:
        w1 = np.zeros((1, 1, 3, 3))
        w1[0, 0, t1 // 3, t1 % 3] = 1.0
        w2 = np.zeros((1, 1, 3, 3))
        w2[0, 0, t2 // 3, t2 % 3] = 2.0
        p = R.flatten([(w1, np.zeros(1)), (w2, np.array([0.5]))])
        net.set_params(p)
        net.forward(xin, out)
        torch.cuda.synchronize()
        ref = R.forward(p, (1, 1, 1), x)[-1]
        assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref), (t1, t2)
