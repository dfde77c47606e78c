"""The allocation-free culling entry point (spamm_cull_noalloc) against the
regular one (spamm_task_list), through the C ABI.

It serves callers that may not allocate device memory (codes that own all of
HBM through their own pool, latency-critical loops that cannot take
cudaMalloc's implicit synchronisation).  Its scratch is one fixed device
array shared by all calls, so the test makes two calls in a row -- a larger
problem, then a smaller one -- and checks that the second does not see the
first one's leftovers.  Task lists are integer results: they must be equal
bit for bit.  This file is named to be collected last."""
import numpy as np
import pytest

from paper_1403_7458_gb300 import synth

pytestmark = pytest.mark.gpu


def _norm_grid(lib, M):
    import torch
    P = 1 << M.depth
    g = torch.empty((P, P), dtype=torch.float64, device="cuda")
    lib.load().spamm_norms(M.handle, M.depth, __import__("ctypes").c_void_p(g.data_ptr()),
                           lib._stream())
    return g


def _run_noalloc(lib, A, B, tau, cap):
    import torch
    nb = A.nb
    off = torch.full((nb * nb + 1,), -7, dtype=torch.int64, device="cuda")
    k = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    lib.cull_noalloc(_norm_grid(lib, A), _norm_grid(lib, B), nb, tau, off, k)
    torch.cuda.synchronize()
    off = off.cpu().numpy()
    total = int(off[-1])
    return off, k.cpu().numpy().view(np.uint32)[:total]


@pytest.mark.parametrize("order", ["large_then_small", "small_then_large"])
def test_noalloc_cull_matches_task_list_two_calls(cuda_lib, order):
    import torch
    cases = [(2048, 32, 1e-6, 11), (640, 32, 1e-4, 12)]
    if order == "small_then_large":
        cases = cases[::-1]
    for n, b, tau, seed in cases:
        a = torch.from_numpy(synth.decaying_matrix(n, seed)).cuda()
        bm = torch.from_numpy(synth.decaying_matrix(n, seed + 1, decay=1.3)).cuda()
        A = cuda_lib.tree_build(a, leaf=b)
        B = cuda_lib.tree_build(bm, leaf=b)
        ref_off, ref_k = cuda_lib.task_list(A, B, tau)
        off, k = _run_noalloc(cuda_lib, A, B, tau, cap=len(ref_k) + 5)
        assert np.array_equal(off, ref_off)
        assert np.array_equal(k, ref_k)


def test_noalloc_rejects_oversize_and_reports_total(cuda_lib):
    import torch
    n2 = torch.ones((1100, 1100), dtype=torch.float64, device="cuda")
    off = torch.zeros((1100 * 1100 + 1,), dtype=torch.int64, device="cuda")
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.cull_noalloc(n2, n2, 1100, 0.0, off, None)
    assert ei.value.status == cuda_lib.E_CAPACITY
    # cap = 0: offsets only, the total tells the caller how much room to give
    a = torch.from_numpy(synth.decaying_matrix(256, 3)).cuda()
    A = cuda_lib.tree_build(a, leaf=32)
    ref_off, _ = cuda_lib.task_list(A, A, 1e-6)
    off = torch.zeros((A.nb * A.nb + 1,), dtype=torch.int64, device="cuda")
    cuda_lib.cull_noalloc(_norm_grid(cuda_lib, A), _norm_grid(cuda_lib, A), A.nb, 1e-6, off, None)
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy(), ref_off)


def test_noalloc_binding_checks_the_tensors(cuda_lib):
    """The binding checks what the C call cannot: device, element type,
    contiguous rows and sizes (a short off or a 2-byte klist would let the
    kernels write past the caller's buffers)."""
    import torch
    nb = 8
    n2 = torch.ones((nb, nb), dtype=torch.float64, device="cuda")
    off = torch.zeros((nb * nb + 1,), dtype=torch.int64, device="cuda")
    k = torch.zeros((16,), dtype=torch.int32, device="cuda")
    bad = [
        (n2.float(), n2, off, k),                                         # float32 norms
        (n2.cpu(), n2, off, k),                                           # host tensor
        (n2[:, :4], n2, off, k),                                          # fewer than nb columns
        (n2.t().contiguous().t()[:, :], n2, off[:-1], k),                 # off too short
        (n2, n2, off, torch.zeros((16,), dtype=torch.int16, device="cuda")),  # 2-byte klist
        (n2, n2, off.int(), k),                                           # int32 offsets
    ]
    for a, b, o, kk in bad:
        with pytest.raises(ValueError):
            cuda_lib.cull_noalloc(a, b, nb, 1e-6, o, kk)
