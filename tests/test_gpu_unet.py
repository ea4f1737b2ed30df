"""The U-Net of the learned warm start against the plain-PyTorch reference (oracle).

BF16 activations and weights with FP32 accumulation against an FP32/FP64
reference: forward within 3e-2 relative L2, parameter gradients within 6e-2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("levels,base,H,B", [(1, 8, 24, 3), (2, 16, 24, 3), (4, 32, 128, 2)])
def test_forward_and_gradients_match_reference(levels, base, H, B):
    from oracle import unet as U
    from paper_2505_08482_gb300.warmstart import UNet
    rng = np.random.default_rng(levels)
    in_ch = 4
    p = U.init_params(levels, base, in_ch, rng)
    x = rng.standard_normal((B, in_ch, H, H)).astype(np.float32)
    t = rng.standard_normal((B, H, H)).astype(np.float32)
    net = UNet(levels, base, in_ch, H, H, max_batch=B)
    assert net.nparam == U.param_count(levels, base, in_ch)
    net.set_params(p)
    # bf16 weights/inputs: compare against the reference evaluated on the bf16-rounded values
    pb = torch.as_tensor(p, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    xb = torch.as_tensor(x).to(torch.bfloat16).double().numpy()
    out = net.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    dt = torch.float64 if H <= 32 else torch.float32
    ref = U.forward(pb, xb, levels, base, in_ch, dtype=dt).detach().numpy()
    assert _rel(out, ref) <= 3e-2
    loss, g = net.grads(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"))
    lref, gref = U.loss_and_grad(pb, xb, t, levels, base, in_ch, dtype=dt)
    assert abs(loss - lref) <= 3e-2 * lref
    assert _rel(g.cpu().numpy(), gref) <= 6e-2


def test_training_reduces_the_loss():
    from oracle import unet as U
    from paper_2505_08482_gb300.warmstart import UNet
    rng = np.random.default_rng(5)
    levels, base, H, B = 3, 16, 32, 8
    net = UNet(levels, base, 4, H, H, max_batch=B)
    net.set_params(U.init_params(levels, base, 4, rng))
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, H), indexing="ij")
    x = rng.standard_normal((B, 4, H, H)).astype(np.float32)
    t = (x[:, 0] * 0.5 + np.tanh(x[:, 1]) * xx).astype(np.float32)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    losses = [float(net.train_step(xd, td, 3e-3).item()) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0]
