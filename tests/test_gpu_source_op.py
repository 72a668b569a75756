"""The surface-to-volume matrix Sbar^E_{i,l} (Section 2, last paragraph) as a
compressed operator on the GPU, against the FP64 oracle's rows of the same
matrix (oracle.source_hat_rows, pinned in test_oracle_pins.py) and against the
library's direct source (rt_source) for a uniform emitter coefficient.

Tolerances: entries are evaluated in FP32 (relative 2e-5 class) and the far
blocks compressed by ACA to a relative Frobenius error of 1e-4, so results are
held to 1e-4 in relative L2 norm."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2306_05789_gb300 as rt
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def run(sop, q, F, N):
    Q = torch.tensor(q, dtype=torch.float32, device=DEV)
    out = torch.full((F, N), float("nan"), dtype=torch.float32, device=DEV)
    sop.apply(Q, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("n,F,R0", [(10, 3, 0.5), (13, 2, 0.0)])
def test_uniform_coefficient_reproduces_the_direct_source(n, F, R0):
    """Q0_l = Q0 for every emitter vertex: sum_l Sbar^E_{i,l} Q0 is the source (the hat
    functions sum to one), so the compressed operator's apply equals rt_source."""
    p = W.cube_problem(n, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3), R0=R0)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    sop = rt.rt_build_source_operator(op)
    try:
        info = sop.info()
        assert info["N"] == p.N and info["L"] == len(O.emitter_vertices(p))
        np.testing.assert_array_equal(sop.vertices, O.emitter_vertices(p))
        y = run(sop, np.full(info["L"], p.Q0), F, p.N)
        src = torch.zeros(F, p.N, dtype=torch.float32, device=DEV)
        op.source(src)
        torch.cuda.synchronize()
        assert rel_l2(y, src.double().cpu().numpy()) < 1e-4
    finally:
        sop.free()
        op.free()


def test_per_vertex_coefficients_match_the_oracle_rows():
    """A non-uniform emitter coefficient: out_nu,i = B_nu(T_emit) sum_l Sbar^E_{g(nu)}[i, l] Q0_l
    against dense FP64 oracle rows of the surface-to-volume matrix on sampled vertices
    (and on every emitter vertex, where the limit values enter)."""
    F = 4
    p = W.cube_problem(16, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams())
    sop = rt.rt_build_source_operator(op)
    try:
        info = sop.info()
        assert info["n_far"] > 0 and info["compression"] > 0.0
        q = np.random.default_rng(21).uniform(0.2, 1.5, info["L"])
        y = run(sop, q, F, p.N)
        sv = O.emitter_vertices(p)
        rows = np.unique(np.concatenate([W.sample_rows(p.N, 120, seed=22), sv[::7]])).astype(np.int32)
        H = O.source_hat_rows(p, rows)              # [r, G, L]
        _, gidx = O.groups_of(p.freqs)
        Bv = O.emitter_intensity(p) / p.Q0
        ref = np.stack([Bv[f] * (H[:, gidx[f], :] @ q) for f in range(F)])
        assert rel_l2(y[:, rows], ref) < 1e-4
    finally:
        sop.free()
        op.free()


def test_grey_problem_and_two_calls_in_a_row():
    """The grey plain-method problem (one channel, sigma T_emit^4) and two applies with
    different coefficients on the same operator (the scratch is reused)."""
    p = W.cube_problem(12, W.Kappa(W.KAPPA_CONST, 1.0, 0.0), W.grey_freqs(), R0=0.5, grey=True)
    op = rt.rt_build_operator(p, rt.hparams())
    sop = rt.rt_build_source_operator(op)
    try:
        L = sop.info()["L"]
        rows = W.sample_rows(p.N, 60, seed=23)
        H = O.source_hat_rows(p, rows)[:, 0, :]
        for seed in (24, 25):
            q = np.random.default_rng(seed).uniform(0.0, 2.0, L)
            y = run(sop, q, 1, p.N)
            ref = O.SIGMA * p.T_emit ** 4 * (H @ q)
            assert rel_l2(y[0, rows], ref) < 1e-4
    finally:
        sop.free()
        op.free()


def test_dense_operator_is_rejected():
    p = W.cube_problem(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    try:
        with pytest.raises(rt.RtError) as e:
            rt.rt_build_source_operator(op)
        assert e.value.code == rt.RT_EINVAL
    finally:
        op.free()


def test_binned_channels_use_their_group_rows():
    """With kappa binning (2 bins for 5 channels) the operator has one N x L matrix per
    bin, built with the bin's midpoint scale; channel f applies its bin's matrix times
    its own intensity: against the oracle's rows at the bins' scales."""
    F = 5
    p = W.cube_problem(12, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(kappa_bins=2))
    sop = rt.rt_build_source_operator(op)
    try:
        info = sop.info()
        assert info["G"] == 2
        q = np.random.default_rng(26).uniform(0.2, 1.5, info["L"])
        y = run(sop, q, F, p.N)
        rows = W.sample_rows(p.N, 80, seed=27)
        cg, gidx = O.groups_of(p.freqs, bins=2)
        H = O.source_hat_rows(p, rows, c=cg)
        Bv = O.emitter_intensity(p) / p.Q0
        ref = np.stack([Bv[f] * (H[:, gidx[f], :] @ q) for f in range(F)])
        assert rel_l2(y[:, rows], ref) < 1e-4
    finally:
        sop.free()
        op.free()
