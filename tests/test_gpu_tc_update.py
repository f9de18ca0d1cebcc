"""tcgen05 trailing update of the mixed-precision LU against a plain PyTorch
reference of the same op (operands rounded to TF32/BF16, FP64 accumulation
in the reference, FP32 accumulation on the tensor cores).  Split modes take
a b as a_hi b_hi + a_hi b_lo + a_lo b_hi."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rnd(x, bf16):
    if bf16:
        return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    # TF32: round to nearest on the 10-bit mantissa
    b = x.to(torch.float32).contiguous().view(torch.int32)
    b = (b + 0x1000) & ~0x1FFF
    return b.view(torch.float32).to(torch.float64)


def _product(L, U, prec):
    bf16 = prec in (2, 4)
    Lh, Uh = _rnd(L, bf16), _rnd(U, bf16)
    if prec in (1, 2):
        return Lh @ Uh
    Ll = _rnd((L - Lh).to(torch.float32).to(torch.float64), bf16)
    Ul = _rnd((U - Uh).to(torch.float32).to(torch.float64), bf16)
    return Lh @ Uh + Lh @ Ul + Ll @ Uh


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(512, 256, 256, 0, 256, 256, 256),     # ld, r0, c0, k0, M, N, Kd
                                   (768, 256, 256, 0, 512, 512, 256),
                                   (768, 352, 352, 320, 416, 32, 32),
                                   (768, 320, 320, 256, 448, 64, 64),
                                   (1024, 384, 384, 256, 640, 128, 128),
                                   (640, 128, 384, 96, 512, 256, 32),
                                   # whole tiles that stop short of the last row (TMA-addressed)
                                   (768, 256, 256, 0, 384, 256, 256),
                                   # ragged tiles inside the matrix (per-thread epilogue)
                                   (768, 260, 256, 0, 300, 200, 64),
                                   # several tiles per persistent CTA (both C and TMEM buffers reused)
                                   (2048, 256, 256, 0, 1792, 1792, 256),
                                   # depth 512 (the merged outer updates of two panels)
                                   (1024, 512, 512, 0, 512, 512, 512)])
def test_trailing_update_matches_torch(prec, shape):
    from paper_2507_22195_gb300 import mehdg
    ld, r0, c0, k0, M, N, Kd = shape
    nK = 3
    g = torch.Generator(device="cuda").manual_seed(1234 + ld + M)
    S = torch.randn((nK, ld, ld), generator=g, device="cuda", dtype=torch.float32)
    # column-major view: T[K][j][i] = S(i, j)  ->  A(i,j) = T[K][j][i]
    A = S.transpose(1, 2).to(torch.float64)
    L = A[:, r0:r0 + M, k0:k0 + Kd]
    U = A[:, k0:k0 + Kd, c0:c0 + N]
    ref = A.clone()
    ref[:, r0:r0 + M, c0:c0 + N] -= _product(L, U, prec)
    scale = (L.abs() @ U.abs()).max().item() + 1.0
    mehdg.mehdg_test_trailing_update(S, r0, c0, k0, M, N, Kd, prec)
    torch.cuda.synchronize()
    out = S.transpose(1, 2).to(torch.float64)
    err = (out - ref).abs().max().item()
    assert err < 2e-6 * scale, (err, scale)
    if prec in (3, 4):
        # the split product is close to the exact FP32 one
        exact = A.clone()
        exact[:, r0:r0 + M, c0:c0 + N] -= L @ U
        assert (out - exact).abs().max().item() < (2e-6 if prec == 3 else 4e-5) * scale
