"""Tensor-core dense kernels of the coarsest direct solve (FP32 cycles).

amg_gemm_tc_f32 (tcgen05 kind::tf32, each operand split into two TF32 parts,
three products per pair) must reach FP32-level accuracy: an error of a few
units of 2^-24 per product plus the FP32 accumulation, far below the 2^-11
relative error of a single TF32 product, which the bound below would reject.
amg_dense_inverse_f32 (blocked LU with partial pivoting, inverse by blocked
triangular solves, every product on the tensor cores) is backward stable: the
inverse's error is at most about c nd u kappa(A), checked against an FP64
inverse, and the CUDA-core path (method 0) meets the same bound.
"""
import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (1, 1, 1), (130, 257, 45), (300, 200, 16), (64, 384, 128),
                                   (1000, 999, 7), (2048, 2048, 16)])
def test_gemm_tc_fp32_accuracy(m, n, k):
    rng = np.random.default_rng(m * 7919 + n * 31 + k)
    a = rng.uniform(-1, 1, (m, k)).astype(np.float32)
    b = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    c = rng.uniform(-1, 1, (m, n)).astype(np.float32)
    cd = dev32(c)
    bamg.amg_gemm_tc_f32(dev32(a), dev32(b), cd)
    torch.cuda.synchronize()
    want = c.astype(np.float64) + a.astype(np.float64) @ b.astype(np.float64)
    got = cd.cpu().numpy().astype(np.float64)
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64) + np.abs(c)
    rel = np.abs(got - want) / scale
    # FP32 accumulation of k products and the final add: (k + 2) u; the split
    # adds about 2^-21 per product; a single TF32 product would show ~2^-11
    assert rel.max() <= (k + 2) * U32 + 2.0 ** -19, rel.max()


def test_gemm_tc_zero_k_and_validation():
    c = np.arange(12, dtype=np.float32).reshape(3, 4)
    cd = dev32(c)
    a = torch.zeros((3, 0), dtype=torch.float32, device="cuda")
    b = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    bamg.amg_gemm_tc_f32(a, b, cd)
    assert np.array_equal(cd.cpu().numpy(), c)
    lib = bamg.load()
    assert lib.amg_gemm_tc_f32(2, 2, 3, None, 2, None, 2, None, 2, None) == bamg.BAMG_EINVAL  # lda < k


def random_matrix(nd, seed, kind):
    rng = np.random.default_rng(seed)
    if kind == "gauss":  # kappa grows like nd
        return rng.standard_normal((nd, nd))
    if kind == "permuted":  # needs pivoting: large entries off the diagonal
        a = rng.uniform(-1, 1, (nd, nd))
        p = rng.permutation(nd)
        a[np.arange(nd), p] += nd
        return a
    raise ValueError(kind)


@pytest.mark.parametrize("nd,kind", [(224, "gauss"), (300, "permuted"), (513, "gauss"), (1014, "permuted"),
                                     (1500, "gauss"), (2048, "gauss")])
@pytest.mark.parametrize("method", [1, 0])
def test_dense_inverse_within_lu_bound(nd, kind, method):
    a = random_matrix(nd, nd, kind).astype(np.float32)
    a64 = a.astype(np.float64)
    inv = torch.empty((nd, nd), dtype=torch.float32, device="cuda")
    ad = dev32(a)
    bamg.amg_dense_inverse_f32(ad, inv, method=method)
    torch.cuda.synchronize()
    assert np.array_equal(ad.cpu().numpy(), a)  # the input is not modified
    got = inv.cpu().numpy().astype(np.float64)
    want = np.linalg.inv(a64)
    kappa = np.linalg.cond(a64, np.inf)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 4.0 * nd * U32 * kappa, (err, kappa)
    # the residual of the inverse, a check independent of the FP64 inverse
    res = np.abs(got @ a64 - np.eye(nd)).max()
    assert res <= 4.0 * nd * U32 * kappa, (res, kappa)


def test_dense_inverse_methods_agree_and_limits():
    nd = 700
    a = random_matrix(nd, 5, "gauss").astype(np.float32)
    outs = []
    for method in (0, 1):
        inv = torch.empty((nd, nd), dtype=torch.float32, device="cuda")
        bamg.amg_dense_inverse_f32(dev32(a), inv, method=method)
        outs.append(inv.cpu().numpy().astype(np.float64))
    kappa = np.linalg.cond(a.astype(np.float64), np.inf)
    assert np.abs(outs[0] - outs[1]).max() / np.abs(outs[0]).max() <= 8.0 * nd * U32 * kappa
    big = torch.zeros((2049, 2049), dtype=torch.float32, device="cuda")
    with pytest.raises(bamg.BamgError) as e:
        bamg.amg_dense_inverse_f32(big, torch.empty_like(big), method=1)
    assert e.value.status == bamg.BAMG_EUNSUPPORTED


@pytest.mark.parametrize("method", [1, 0])
def test_dense_inverse_singular(method):
    nd = 400
    a = random_matrix(nd, 9, "gauss")
    a[:, 17] = 0.0  # a zero column: no pivot for it
    inv = torch.empty((nd, nd), dtype=torch.float32, device="cuda")
    with pytest.raises(bamg.BamgError) as e:
        bamg.amg_dense_inverse_f32(dev32(a), inv, method=method)
    assert e.value.status == bamg.BAMG_ESINGULAR_COARSE
