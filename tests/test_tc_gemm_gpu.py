"""The mixed-precision trailing update (tcgen05 tensor-core kernel and its SIMT
twin) against an exact reference: products of the 16-bit operands summed in
float64 on the host.  Both kernels accumulate in FP32, so the bound is the
FP32 summation error, K * 2^-24 * sum_k |a_ik b_jk| (plus the FP32 rounding of
C itself)."""
import numpy as np
import pytest
import torch

import paper_1907_05767_gb300 as ebv

pytestmark = pytest.mark.gpu


def run_case(m0, n0, k0, M, N, K, ld, dtype, engine, seed=0, scale=(1.0, 1.0), cpad=5):
    g = torch.Generator().manual_seed(seed)
    rows = max(m0 + M, n0 + N) + 3
    lb = (torch.rand((rows, ld), generator=g, dtype=torch.float64) - 0.5).to(dtype)
    ut = (torch.rand((rows, ld), generator=g, dtype=torch.float64) - 0.5).to(dtype)
    c0 = torch.rand((rows, n0 + N + cpad), generator=g, dtype=torch.float32)
    s = torch.tensor([scale[0], scale[1], 1.0 / (scale[0] * scale[1]), 0.0], dtype=torch.float32)
    c = c0.clone().cuda()
    ebv.debug_lowp_update(c, lb.cuda(), ut.cuda(), s.cuda(), m0, n0, k0, M, N, K, engine)
    got = c.cpu().double()
    a = lb[m0:m0 + M, k0:k0 + K].double()
    b = ut[n0:n0 + N, k0:k0 + K].double()
    ref = c0.double().clone()
    ref[m0:m0 + M, n0:n0 + N] -= (a @ b.T) * float(s[2])
    bound = K * 2.0 ** -24 * ((a.abs() @ b.abs().T) * float(s[2])) + 2.0 ** -23 * ref[m0:m0 + M, n0:n0 + N].abs()
    diff = (got - ref).abs()
    inside = diff[m0:m0 + M, n0:n0 + N]
    assert torch.all(inside <= bound + 1e-30), float((inside - bound).max())
    # nothing outside the target block changes
    mask = torch.ones_like(diff, dtype=torch.bool)
    mask[m0:m0 + M, n0:n0 + N] = False
    assert torch.all(diff[mask] == 0)


@pytest.mark.parametrize("engine", ["simt", "tc"])
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("shape", [
    (0, 0, 0, 128, 256, 64),      # one tile, one K slab
    (0, 0, 0, 256, 512, 256),     # several tiles and slabs (ring reuse)
    (64, 128, 64, 300, 200, 640), # ragged M, N (BN 256 path), K over 10 slabs
    (5, 64, 128, 129, 100, 192),  # ragged, BN 128
    (0, 0, 0, 1000, 64, 64),      # tall and narrow, BN 64
    (128, 64, 0, 77, 33, 128),    # small ragged block
])
def test_lowp_update_exact_reference(engine, dtype, shape):
    m0, n0, k0, M, N, K = shape
    ld = ((k0 + K + 63) // 64) * 64 + 64
    run_case(m0, n0, k0, M, N, K, ld, dtype, engine)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("shape", [
    (0, 0, 0, 256, 256, 256),      # whole tiles, four slabs (one ring)
    (64, 128, 64, 300, 200, 448),  # ragged M and N, seven slabs (ring reuse)
    (5, 64, 128, 129, 100, 192),   # ragged, three slabs (fewer than the ring)
    (128, 64, 0, 77, 72, 128),     # one partial tile
    (0, 0, 0, 640, 384, 512),      # the largest K of the small-K kernel
])
def test_tc_small_k_c_in_shared_memory(dtype, shape):
    # 16-byte rows of C (width a multiple of 4): K <= 512 and N > 64 take the
    # kernel that stages C in shared memory and stores it back by TMA; the
    # block edges must clip (nothing outside the block changes).
    m0, n0, k0, M, N, K = shape
    ld = ((k0 + K + 63) // 64) * 64 + 64
    cpad = 4 + (-(n0 + N)) % 4
    run_case(m0, n0, k0, M, N, K, ld, dtype, "tc", cpad=cpad)


def test_tc_scaled_half():
    run_case(0, 0, 0, 256, 256, 128, 192, torch.float16, "tc", scale=(2.0 ** 10, 2.0 ** 12))


def test_tc_equals_simt_bitwise_on_exact_products():
    # Small-integer operands: every product and every partial sum is exact in
    # FP32, so the two engines (any summation order) agree bit for bit.
    g = torch.Generator().manual_seed(3)
    M, N, K, ld = 256, 256, 256, 256
    lb = torch.randint(-8, 9, (M, ld), generator=g).to(torch.bfloat16)
    ut = torch.randint(-8, 9, (N, ld), generator=g).to(torch.bfloat16)
    s = torch.tensor([1.0, 1.0, 1.0, 0.0]).cuda()
    c1 = torch.zeros((M, N), dtype=torch.float32).cuda()
    c2 = c1.clone()
    ebv.debug_lowp_update(c1, lb.cuda(), ut.cuda(), s, 0, 0, 0, M, N, K, "tc")
    ebv.debug_lowp_update(c2, lb.cuda(), ut.cuda(), s, 0, 0, 0, M, N, K, "simt")
    ref = -(lb.double() @ ut.double().T).float()
    assert torch.equal(c1.cpu(), ref) and torch.equal(c2.cpu(), ref)


def test_tc_rejects_unaligned_k():
    c = torch.zeros((128, 128), dtype=torch.float32).cuda()
    lb = torch.zeros((128, 128), dtype=torch.bfloat16).cuda()
    s = torch.tensor([1.0, 1.0, 1.0, 0.0]).cuda()
    with pytest.raises(ebv.EbvError) as e:
        ebv.debug_lowp_update(c, lb, lb, s, 0, 0, 0, 128, 128, 96, "tc")
    assert e.value.status == ebv.ERR_UNSUPPORTED
