"""Kernel-level checks of the tensor-core product (with its fused epilogue)
and of the BF16 split, against plain PyTorch float64 references computed
from the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def padded(rows, cols, dtype, fill=0.0):
    import torch
    ld = (cols + 7) // 8 * 8
    return torch.full((rows, ld), fill, dtype=dtype, device="cuda")[:, :cols]


def split(x):
    import torch
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    return hi, lo


def to_dev_bf16(t):
    import torch
    d = padded(t.shape[0], t.shape[1], torch.bfloat16)
    d.copy_(t.cuda())
    return d


def product(ah, al, bh, bl, nsplit):
    ref = ah.double() @ bh.double().T
    if nsplit == 3:
        ref = ref + ah.double() @ bl.double().T + al.double() @ bh.double().T
    return ref


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 256), (200, 136, 72), (1, 1, 1), (130, 300, 520),
                                   (1024, 1024, 1024), (384, 2048, 64), (4096, 1000, 200)])
@pytest.mark.parametrize("nsplit", [1, 3])
def test_general_product(lib, M, N, K, nsplit):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 13 + K)
    ah, al = split(torch.randn((M, K), generator=g))
    bh, bl = split(torch.randn((N, K), generator=g))
    D = torch.full((M, N), float("nan"), device="cuda")
    lib.kernel_gemm_bf16(to_dev_bf16(ah), to_dev_bf16(al), to_dev_bf16(bh), to_dev_bf16(bl), nsplit, D, diag=0.5)
    torch.cuda.synchronize()
    ref = product(ah, al, bh, bl, nsplit) + 0.5 * torch.eye(M, N, dtype=torch.float64)
    err = (D.cpu().double() - ref).abs().max().item()
    assert err <= 1e-5 * (1 + ref.abs().max().item()) * max(1, K) ** 0.5, err


@pytest.mark.parametrize("p,K", [(64, 64), (256, 256), (300, 300), (1000, 1000), (130, 70), (2048, 2048)])
@pytest.mark.parametrize("nsplit", [1, 3])
def test_symmetric_recurrence_step(lib, p, K, nsplit):
    """One fused step: v = 2 acc - C - 2 C2 - Id, D = v and H += c_k v in the
    lower triangle, BF16 hi/lo of v in both triangles."""
    import torch
    g = torch.Generator().manual_seed(p * 31 + K)
    S = torch.randn((p, K), generator=g) / K ** 0.5
    Af = S            # A B^T = S S^T is symmetric
    Bf = S.clone()
    ah, al = split(Af)
    bh, bl = split(Bf)
    Cm = torch.randn((p, p), generator=g); Cm = (Cm + Cm.T) / 2
    C2m = torch.randn((p, p), generator=g); C2m = (C2m + C2m.T) / 2
    Hm = torch.randn((p, p), generator=g); Hm = (Hm + Hm.T) / 2
    C, C2, H = padded(p, p, torch.float32), padded(p, p, torch.float32), padded(p, p, torch.float32)
    C.copy_(Cm.cuda()); C2.copy_(C2m.cuda()); H.copy_(Hm.cuda())
    D = C   # in place over C, as the recurrence does
    coef = torch.tensor([0.0, 0.0, 0.0, 0.125], dtype=torch.float64, device="cuda")
    Dhi, Dlo = padded(p, p, torch.bfloat16), padded(p, p, torch.bfloat16)
    lib.kernel_gemm_bf16(to_dev_bf16(ah), to_dev_bf16(al), to_dev_bf16(bh), to_dev_bf16(bl), nsplit, D, sym=True,
                         s_acc=2.0, C=C, s_c=-1.0, C2=C2, s_c2=-2.0, diag=-1.0, H=H, coef=coef, k=3,
                         Dhi=Dhi, Dlo=Dlo)
    torch.cuda.synchronize()
    acc = product(ah, al, bh, bl, nsplit)
    v = 2 * acc - Cm.double() - 2 * C2m.double() - torch.eye(p, dtype=torch.float64)
    # the kernel takes the upper-triangle value of the product for both positions
    vu = torch.triu(v) + torch.triu(v, 1).T
    low = torch.tril(torch.ones(p, p, dtype=torch.bool))
    tol = 1e-5 * (1 + vu.abs().max().item()) * K ** 0.5
    Dg = D.cpu().double()
    assert (Dg - vu)[low].abs().max().item() <= tol
    Hg = H.cpu().double()
    assert (Hg - (Hm.double() + 0.125 * vu))[low].abs().max().item() <= tol
    hi = Dhi.cpu().float()
    assert torch.allclose(hi.double(), vu, rtol=2 ** -8, atol=tol)
    assert torch.equal(hi, hi.T)   # both triangles, exactly symmetric
    # hi/lo pair: lower triangle equals the split of the stored FP32 value
    h_ref, l_ref = split(D.cpu())
    assert torch.equal(Dhi.cpu()[low], h_ref[low]) and torch.equal(Dlo.cpu()[low], l_ref[low])


@pytest.mark.parametrize("rows,cols", [(64, 64), (100, 37), (1, 9), (257, 129)])
@pytest.mark.parametrize("transpose", [False, True])
def test_split_bf16(lib, rows, cols, transpose):
    import torch
    X = torch.randn((rows, cols), device="cuda")
    r, c = (cols, rows) if transpose else (rows, cols)
    hi = padded(r, c, torch.bfloat16)
    lo = padded(r, c, torch.bfloat16)
    lib.kernel_split_bf16(X, transpose, hi, lo)
    torch.cuda.synchronize()
    Xr = X.T if transpose else X
    h = Xr.cpu().to(torch.bfloat16)
    assert torch.equal(hi.cpu(), h)
    assert torch.equal(lo.cpu(), (Xr.cpu() - h.float()).to(torch.bfloat16))


@pytest.mark.parametrize("p", [1, 7, 64, 300, 1024])
def test_topk_eps_is_the_kth_largest_magnitude(lib, p):
    """The entry threshold of the top-k mode (Eq. recommendation_epsilon's
    K(|Phi|, k)): the k-th largest |Phi_ij| exactly, bit for bit against
    numpy's sort, with ties, signed zeros, subnormals and a padded row
    stride, for k = 1, p^2 and values between."""
    import torch
    rng = np.random.default_rng(p)
    Phi = rng.standard_normal((p, p)).astype(np.float32) * np.exp(rng.uniform(-30, 30, (p, p))).astype(np.float32)
    flat = Phi.ravel()
    flat[rng.integers(0, flat.size, size=max(1, flat.size // 5))] = 0.0        # exact zeros
    flat[rng.integers(0, flat.size, size=max(1, flat.size // 7))] = -0.0
    flat[rng.integers(0, flat.size, size=max(1, flat.size // 9))] = 3.25         # ties
    flat[rng.integers(0, flat.size, size=max(1, flat.size // 11))] = 1e-40       # subnormal
    Phi = flat.reshape(p, p)
    ld = p + 5
    dev = torch.zeros((p, ld), dtype=torch.float32, device="cuda")
    dev[:, p:] = 1e30   # padding beyond p must not be read
    dev[:, :p] = torch.from_numpy(Phi).cuda()
    srt = np.sort(np.abs(Phi).ravel())[::-1]
    for k in sorted(k for k in {1, 2, max(1, p * p // 3), max(1, p * p // 2), p * p} if k <= p * p):
        got = lib.kernel_topk_eps(dev[:, :p], k)
        assert np.float32(got).view(np.uint32) == np.float32(srt[k - 1]).view(np.uint32), (p, k, got, srt[k - 1])
    with pytest.raises(lib.CpaError):
        lib.kernel_topk_eps(dev[:, :p], p * p + 1)
