"""hss_gemm_f32_static (the FP32 GEMM with its launch records in the library's
fixed device array, no allocation in the call) against hss_gemm_f32, through
the C ABI.  Named to be collected last, so it also runs after every other
test has used the library (and its allocating workspace) in this process."""
import ctypes

import pytest


def _hss():
    import __graft_entry__ as g
    g.build()
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def test_static_gemm_rejects_more_tiles_than_the_scratch_holds():
    """The size check runs on the host before any device work: 8192 x 8256
    needs 128 x 129 tiles of 64 x 64, one column of tiles over the limit."""
    hs = _hss()
    lib = hs._lib
    fake = ctypes.c_void_p(256)   # never dereferenced: the call returns at the size check
    m, n, k = 8192, 8256, 16
    rc = lib.hss_gemm_f32_static(m, n, k, fake, m, fake, k, fake, m, 1.0, 0.0, 0, None)
    assert rc == hs.HSS_EINVAL
    msg = lib.hss_last_error().decode()
    assert "16512 tiles" in msg and str(hs.GEMM_STATIC_MAX_TILES) in msg
    rc = lib.hss_gemm_f32_static(m, n, k, fake, m, fake, k, fake, m, 1.0, 0.0, 3, None)
    assert rc == hs.HSS_EINVAL and "invalid argument" in lib.hss_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("engine,tol", [(0, 2e-6), (1, 2e-6), (2, 2e-3)])
def test_static_gemm_matches_allocating_gemm_two_calls_in_a_row(engine, tol):
    """Two consecutive calls with different shapes, data, alpha and beta: each
    agrees with hss_gemm_f32 on the same inputs (and with an FP64 product), so
    the second call reads its own records, not the first call's."""
    import torch
    hs = _hss()
    g = torch.Generator(device="cpu").manual_seed(1508 + engine)
    cases = [((300, 200, 130), 0.5, 2.0), ((129, 513, 257), -1.0, 0.25)]
    for (m, n, k), alpha, beta in cases:
        A = torch.randn(m, k, generator=g).cuda()
        B = torch.randn(k, n, generator=g).cuda()
        C0 = torch.randn(m, n, generator=g).cuda()
        ref = (A.double() @ B.double()) * alpha + C0.double() * beta
        scale = abs(alpha) * (A.double().abs() @ B.double().abs()).max().item() + abs(beta) * C0.abs().max().item()
        Cs = C0.clone()
        Ca = C0.clone()
        torch.cuda.synchronize()
        hs.gemm_f32_static(A, B, Cs, alpha=alpha, beta=beta, engine=engine)
        hs.gemm_f32(A, B, Ca, alpha=alpha, beta=beta, engine=engine)
        torch.cuda.synchronize()
        d_alloc = (Cs.double() - Ca.double()).abs().max().item() / scale
        d_ref = (Cs.double() - ref).abs().max().item() / scale
        assert d_alloc <= tol, (engine, (m, n, k), d_alloc)
        assert d_ref <= tol, (engine, (m, n, k), d_ref)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", [0, 1, 2])
def test_static_gemm_allocates_nothing(engine):
    """The property the entry point exists for: after one warm-up call (which
    does the per-device setup) a call makes no memory request of any kind --
    the library's request counter and the device's free memory are the same
    before and after it -- while hss_gemm_f32 on the same operands does make
    requests (its workspace), so the counter does see them."""
    import torch
    hs = _hss()
    g = torch.Generator(device="cpu").manual_seed(11 + engine)
    m, n, k = 300, 260, 140
    A = torch.randn(m, k, generator=g).cuda()
    B = torch.randn(k, n, generator=g).cuda()
    C = torch.zeros(m, n, device="cuda")
    Ca = torch.zeros(m, n, device="cuda")
    hs.gemm_f32_static(A, B, C, engine=engine)          # warm-up: per-device setup
    torch.cuda.synchronize()
    a0 = hs.alloc_count()
    free0 = torch.cuda.mem_get_info()[0]
    hs.gemm_f32_static(A, B, C, alpha=0.5, beta=0.5, engine=engine)
    torch.cuda.synchronize()
    assert hs.alloc_count() == a0
    assert torch.cuda.mem_get_info()[0] == free0
    hs.gemm_f32(A, B, Ca, engine=engine)
    assert hs.alloc_count() > a0
    ref = (A.double() @ B.double()) * 0.5 + 0.5 * (A.double() @ B.double())
    scale = (A.double().abs() @ B.double().abs()).max().item()
    assert (C.double() - ref).abs().max().item() / scale <= (2e-3 if engine == 2 else 2e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", [0, 1, 2])
def test_k_zero_gives_beta_c(engine):
    """k = 0: C = beta C for every engine in both entry points (no product;
    the tensor-core engines must not read an accumulator nothing wrote)."""
    import torch
    hs = _hss()
    lib = hs._lib
    g = torch.Generator(device="cpu").manual_seed(5)
    m, n = 200, 150
    dummy = torch.zeros(4, device="cuda")   # A and B are never read when k = 0
    for fn in (lib.hss_gemm_f32, lib.hss_gemm_f32_static):
        for beta in (0.0, -1.5):
            C0 = torch.randn(n, m, generator=g).cuda()   # column-major m x n
            C = C0.clone()
            rc = fn(m, n, 0, ctypes.c_void_p(dummy.data_ptr()), m, ctypes.c_void_p(dummy.data_ptr()), 1,
                    ctypes.c_void_p(C.data_ptr()), m, 2.0, beta, engine, None)
            torch.cuda.synchronize()
            assert rc == hs.HSS_OK, lib.hss_last_error()
            assert torch.equal(C, C0 * beta) if beta != 0.0 else torch.count_nonzero(C).item() == 0


@pytest.mark.gpu
def test_static_gemm_at_the_tile_limit():
    """m = n = 8192 with the SIMT engine fills all 16384 tile slots."""
    import torch
    hs = _hss()
    g = torch.Generator(device="cpu").manual_seed(7)
    m = n = 8192
    k = 32
    A = torch.randn(m, k, generator=g).cuda()
    B = torch.randn(k, n, generator=g).cuda()
    Cs = torch.zeros(m, n, device="cuda")
    Ca = torch.zeros(m, n, device="cuda")
    hs.gemm_f32_static(A, B, Cs, engine=0)
    hs.gemm_f32(A, B, Ca, engine=0)
    torch.cuda.synchronize()
    scale = (A.abs() @ B.abs()).max().item()
    assert (Cs - Ca).abs().max().item() / scale <= 2e-6
    # spot rows against FP64
    rows = torch.tensor([0, 1, 4095, 8191], device="cuda")
    ref = A[rows].double() @ B.double()
    assert (Cs[rows].double() - ref).abs().max().item() / scale <= 2e-6
