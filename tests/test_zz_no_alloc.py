"""The allocation-free L1 entry point (for callers that cannot allocate
device memory) against the allocating one, through the C ABI.  Collected
last on purpose: it runs after every other test, and also alone."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_06161_gb300 import _lib

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4  # the feature tolerance of the parity tests (sums regroup)


def _pair(seed, rows, ch):
    rng = np.random.default_rng(seed)
    pred = torch.as_tensor(rng.normal(size=(rows, ch)).astype(np.float32), device="cuda")
    tgt = torch.as_tensor(rng.normal(size=(rows, ch)).astype(np.float32), device="cuda")
    return pred, tgt


def test_noalloc_l1_matches_allocating_entry_point_twice():
    for seed, (rows, ch) in enumerate([(640 * 512, 32), (640 * 512, 3)]):
        pred, tgt = _pair(seed, rows, ch)
        g_ref = torch.empty_like(pred)
        l_ref = torch.zeros(1, device="cuda")
        scratch = torch.empty(1024, device="cuda")
        _lib.fe_l1_loss_grad(pred, tgt, rows, g_ref, l_ref, scratch)
        g = torch.full_like(pred, float("nan"))
        l = torch.full((1,), float("nan"), device="cuda")
        _lib.fe_l1_loss_grad_noalloc(pred, tgt, rows, g, l)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
        a, b = float(l.item()), float(l_ref.item())
        assert abs(a - b) <= REL_TOL * abs(b), (a, b)


@pytest.mark.parametrize("rows,ch,offset", [(640 * 512 + 1, 3, 0), (1000, 3, 1), (5, 1, 0)])
def test_noalloc_l1_tail_and_unaligned_inputs(rows, ch, offset):
    # n not a multiple of 4 (scalar tail) and inputs one float past a 16-byte
    # boundary (the scalar path throughout), against the allocating entry point.
    rng = np.random.default_rng(rows + offset)
    n = rows * ch
    base_p = torch.as_tensor(rng.normal(size=n + offset).astype(np.float32), device="cuda")
    base_t = torch.as_tensor(rng.normal(size=n + offset).astype(np.float32), device="cuda")
    pred, tgt = base_p[offset:], base_t[offset:]
    base_g = torch.empty(n + offset, device="cuda")
    g = base_g[offset:]
    g_ref = torch.empty(n, device="cuda")
    l_ref = torch.zeros(1, device="cuda")
    _lib.fe_l1_loss_grad(pred, tgt, rows, g_ref, l_ref, torch.empty(1024, device="cuda"))
    for _ in range(2):
        g.fill_(float("nan"))
        l = torch.full((1,), float("nan"), device="cuda")
        _lib.fe_l1_loss_grad_noalloc(pred, tgt, rows, g, l)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
        a, b = float(l.item()), float(l_ref.item())
        assert abs(a - b) <= REL_TOL * abs(b), (a, b)


def test_noalloc_l1_rejects_sizes_past_its_array():
    L = _lib.load()
    x = torch.zeros(4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    too_many = 16384 * 2048 + 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.fe_l1_loss_grad_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), too_many, 1,
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(loss.data_ptr()), stream)
    assert rc == 3  # FE_ERR_WORKSPACE: nothing launched
