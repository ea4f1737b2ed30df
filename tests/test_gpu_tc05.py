"""The BF16 GEMM on the fifth-generation tensor cores (tcgen05.mma with the accumulator in
tensor memory, operands copied by TMA) against the warp-level GEMM and an FP64 product.

The operands are BF16 (exact in FP64), the products are exact in FP32 and the sums
accumulate in FP32, so both paths agree with the FP64 product of the BF16 inputs to
a few FP32 roundings per term: the bound below is 1e-5 of sum |a||b| per entry.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gemm(A, B, path, status=None):
    from paper_2505_08482_gb300 import _binding as Bd
    M, K = A.shape
    N = B.shape[0]
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = Bd.lib().pat_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                                B.stride(0), M, N, K, ctypes.c_void_p(C.data_ptr()), N, path,
                                ctypes.c_void_p(status.data_ptr()) if status is not None else None, st)
    assert rc == Bd.PAT_OK, Bd.lib().pat_last_error()
    return C


# the last shape has enough tiles for the 256-wide N tile (ragged in M, N and K)
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 72, 136), (1000, 256, 576), (4096, 32, 72),
                                   (64, 300, 4608), (20000, 300, 136)])
def test_tc05_gemm_matches_fp64_and_warp_path(M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    C1 = _gemm(A, B, 1, status)
    C0 = _gemm(A, B, 0)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a, b = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = a @ b.T
    bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(C1.cpu().numpy() - ref) <= bound)
    assert np.all(np.abs(C0.cpu().numpy() - ref) <= bound)


def test_tc05_rejects_operands_the_tma_cannot_address():
    from paper_2505_08482_gb300 import _binding as Bd
    A = torch.zeros((128, 32), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    rc = Bd.lib().pat_gemm_bf16(ctypes.c_void_p(A.data_ptr()), 32, ctypes.c_void_p(A.data_ptr()), 32, 128, 128, 32,
                                ctypes.c_void_p(C.data_ptr()), 128, 1, None, None)
    assert rc == Bd.PAT_EINVAL


@pytest.mark.parametrize("levels,base,H,B", [(2, 16, 24, 3), (4, 32, 128, 2)])
def test_unet_on_tc05_matches_warp_path_and_reference(levels, base, H, B):
    from oracle import unet as U
    from paper_2505_08482_gb300.warmstart import UNet
    rng = np.random.default_rng(levels + 10)
    in_ch = 4
    p = U.init_params(levels, base, in_ch, rng)
    x = torch.as_tensor(rng.standard_normal((B, in_ch, H, H)).astype(np.float32), device="cuda")
    t = torch.as_tensor(rng.standard_normal((B, H, H)).astype(np.float32), device="cuda")
    out = {}
    for path in (0, 1):
        net = UNet(levels, base, in_ch, H, H, max_batch=B)
        net.set_params(p)
        net.gemm_path = path
        y = net.forward(x).cpu().numpy()
        loss, g = net.grads(x, t)
        assert net.status() == 0
        out[path] = (y, loss, g.cpu().numpy())
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    # both paths round the same FP32 sums to BF16 activations: close, not equal
    assert rel(out[1][0], out[0][0]) <= 1e-2
    assert rel(out[1][2], out[0][2]) <= 2e-2
    pb = torch.as_tensor(p, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    xb = x.cpu().to(torch.bfloat16).double().numpy()
    dt = torch.float64 if H <= 32 else torch.float32
    ref = U.forward(pb, xb, levels, base, in_ch, dtype=dt).detach().numpy()
    assert rel(out[1][0], ref) <= 3e-2
    lref, gref = U.loss_and_grad(pb, xb, t.cpu().numpy(), levels, base, in_ch, dtype=dt)
    assert abs(out[1][1] - lref) <= 3e-2 * lref
    assert rel(out[1][2], gref) <= 6e-2
