"""The allocation-free gradient entry point (amr_mlp_grad_noalloc).

It serves callers that cannot allocate device memory: code inside a
task-based runtime that owns all device memory, and real-time loops where an
allocation could synchronise the device. Its result must equal the allocating
entry point (amr_mlp_grad) on the same inputs, call after call, although its
hidden activations live in one fixed array shared by every call.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def cuda():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def inputs(seed, n, dim):
    from paper_2508_05020_gb300 import amr
    rng = np.random.default_rng(seed)
    K = amr.mlp_k(dim)
    X = rng.normal(0.0, 0.3, size=(n, K)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.2).astype(np.float32)
    lim1, lim2 = np.sqrt(6.0 / K), np.sqrt(6.0 / 64)
    w = np.concatenate([rng.uniform(-lim1, lim1, 64 * K), np.zeros(64), rng.uniform(-lim2, lim2, 64 * 64),
                        np.zeros(64), rng.uniform(-lim2, lim2, 64) * 0.5, np.zeros(1)]).astype(np.float32)
    pw = float((n - y.sum()) / max(y.sum(), 1.0))
    return X, y, w, pw


def noalloc_grad(dim, X, y, w, pw):
    import torch
    from paper_2508_05020_gb300 import amr
    lib = amr.load()
    dX = torch.from_numpy(X).cuda()
    dy = torch.from_numpy(y).cuda()
    dw = torch.from_numpy(w).cuda()
    dg = torch.full((w.size,), float('nan'), dtype=torch.float32, device='cuda')
    dl = torch.full((1,), float('nan'), dtype=torch.float32, device='cuda')
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.amr_mlp_grad_noalloc(dim, C.c_void_p(dX.data_ptr()), C.c_void_p(dy.data_ptr()), X.shape[0],
                                  C.c_float(pw), C.c_void_p(dw.data_ptr()), C.c_void_p(dg.data_ptr()),
                                  C.c_void_p(dl.data_ptr()), C.c_void_p(stream))
    torch.cuda.synchronize()
    assert rc == 0, rc
    return float(dl.cpu()[0]), dg.cpu().numpy()


@pytest.mark.parametrize('dim', [1, 2, 3])
def test_noalloc_gradient_equals_allocating_call_twice(dim):
    from paper_2508_05020_gb300 import amr
    # two calls in a row: the second uses fewer rows, so stale rows of the
    # first call are still in the shared array
    for seed, n in ((11, 1500), (12, 700)):
        X, y, w, pw = inputs(seed, n, dim)
        l_ref, g_ref = amr.mlp_grad(dim, X, y, pw, w)
        l_na, g_na = noalloc_grad(dim, X, y, w, pw)
        assert abs(l_na - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
        assert np.linalg.norm(g_na - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_noalloc_rejects_more_rows_than_its_scratch():
    import torch
    from paper_2508_05020_gb300 import amr
    lib = amr.load()
    n = 2049
    dX = torch.zeros((n, amr.mlp_k(1)), dtype=torch.float32, device='cuda')
    dy = torch.zeros(n, dtype=torch.float32, device='cuda')
    dw = torch.zeros(amr.mlp_k(1) * 64 + 64 + 4096 + 64 + 64 + 1, dtype=torch.float32, device='cuda')
    dg = torch.zeros_like(dw)
    dl = torch.zeros(1, dtype=torch.float32, device='cuda')
    rc = lib.amr_mlp_grad_noalloc(1, C.c_void_p(dX.data_ptr()), C.c_void_p(dy.data_ptr()), n, C.c_float(1.0),
                                  C.c_void_p(dw.data_ptr()), C.c_void_p(dg.data_ptr()), C.c_void_p(dl.data_ptr()),
                                  None)
    assert rc == -1                    # AMR_ERR_ARG
