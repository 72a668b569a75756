"""rt_apply_noalloc: the operator apply for callers that must not allocate.

Some callers cannot call cudaMalloc while they run: an application whose
device memory is entirely handed out by its own pool allocator, or a host loop
with a fixed time budget that cannot afford the synchronisation an allocation
or a free may imply.  For them rt_apply_noalloc takes its scratch from a static
device array of the library instead of allocating.  This file is collected
last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2306_05789_gb300 as rt
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_05789_gb300 import build
    build.build()


def test_noalloc_apply_matches_rt_apply_on_two_calls_in_a_row():
    p = W.cube_problem(10, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    for seed in (0, 1):   # two calls in a row, different inputs, same scratch array
        X = torch.tensor(W.rand_vectors((3, p.N), seed=seed), dtype=torch.float32, device=DEV)
        Y_ref = torch.zeros_like(X)
        Y = torch.full_like(X, float("nan"))
        op.apply(X, Y_ref)
        op.apply_noalloc(X, Y)
        torch.cuda.synchronize()
        ref = Y_ref.cpu().numpy()
        got = Y.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    op.free()


def test_noalloc_apply_dense_operator():
    p = W.cube_problem(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    X = torch.tensor(W.rand_vectors((2, p.N), seed=2), dtype=torch.float64, device=DEV)
    Y_ref = torch.zeros_like(X)
    Y = torch.zeros_like(X)
    op.apply(X, Y_ref)
    op.apply_noalloc(X, Y)
    op.apply_noalloc(X, Y)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Y.cpu().numpy(), Y_ref.cpu().numpy(), rtol=1e-12)
    op.free()


def test_noalloc_apply_rejects_operators_beyond_the_scratch_limit():
    p = W.multifreq_32(n=24, F=16)
    op = rt.rt_build_operator(p, rt.hparams())
    X = torch.rand(16, p.N, device=DEV)
    Y = torch.zeros_like(X)
    with pytest.raises(rt.RtError) as e:
        op.apply_noalloc(X, Y)
    assert e.value.code == rt.RT_EINVAL
    assert "limit" in str(e.value)
    op.free()


def test_noalloc_apply_takes_the_tensor_core_path_like_rt_apply():
    """A BF16 far field with one operator for 16 right-hand sides: rt_apply runs the
    tcgen05 pair, and so does the no-allocation entry (same kernels, same result)."""
    F = 16
    p = W.cube_problem(10, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3, c_offset=None), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32, far_prec=rt.RT_PREC_BF16))
    assert op.info()["apply_tensor_cores"] == 1
    for seed in (3, 4):
        X = torch.tensor(W.rand_vectors((F, p.N), seed=seed), dtype=torch.float32, device=DEV)
        Y_ref = torch.zeros_like(X)
        Y = torch.full_like(X, float("nan"))
        op.apply(X, Y_ref)
        op.apply_noalloc(X, Y)
        torch.cuda.synchronize()
        ref = Y_ref.cpu().numpy()
        got = Y.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    op.free()


def test_noalloc_apply_leaves_free_device_memory_unchanged():
    """After the first call (which looks up the array's address), further calls change
    neither the device's free memory nor the result."""
    p = W.cube_problem(10, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    X = torch.tensor(W.rand_vectors((3, p.N), seed=5), dtype=torch.float32, device=DEV)
    Y0 = torch.zeros_like(X)
    Y = torch.zeros_like(X)
    op.apply_noalloc(X, Y0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        op.apply_noalloc(X, Y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(Y, Y0)
    op.free()
