"""Ragged batch of independent problems (sipg_batch_*): every member's
solution against the oracle's exact global fast-diagonalisation solve and
against the same problem solved alone; the full 64-problem 2D batch (2^L x 2^L
cells, L in 5..9, degree 2..6) as the benchmark runs it.  With
SIPG_BATCH_FUSED=1 all-2D FP32 batches take the fused path (one cooperative
launch per smoothing stage across the members, one CUDA graph per FCG
iteration of the batch): its members match the oracle's exact solves and the
same batch on the per-member path, including the full 64-problem batch."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from oracle.direct import GlobalFD  # noqa: E402
from paper_2405_18982_gb300 import SIPG, SIPG_FP32, SIPG_FP64, Params, SIPGBatch, SipgError, inputs  # noqa: E402


def _params(shapes, prec, graphs=1):
    return [Params(dim=d, degree=k, log2_cells=L, n_levels=L, vcycle_precision=prec, use_graphs=graphs)
            for d, L, k in shapes]


def _rhs(batch, seed0):
    return [dev(inputs.normal(seed0 + i, m.ndofs())) for i, m in enumerate(batch.members)]


SMALL = [(2, 3, 1), (2, 5, 6), (2, 4, 3), (3, 2, 2), (2, 6, 2), (3, 3, 4), (2, 2, 7), (2, 5, 4)]


@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "mixed"])
def test_small_ragged_batch_matches_direct_and_single(prec):
    import torch
    bt = SIPGBatch(_params(SMALL, prec))
    bs = _rhs(bt, 300)
    xs = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, rtol=1e-10, maxit=100)
    for (d, L, k), b, x, inf in zip(SMALL, bs, xs, infos):
        assert inf.status == 0 and inf.rel_residual <= 1e-10
        u = GlobalFD(d, k, 1 << L).solve(host(b))
        err = np.linalg.norm(host(x) - u) / np.linalg.norm(u)
        assert err < (1e-8 if prec == SIPG_FP32 else 1e-9), (d, L, k, err)
        alone = SIPG(Params(dim=d, degree=k, log2_cells=L, n_levels=L, vcycle_precision=prec, use_graphs=1))
        xa = torch.zeros_like(b)
        ia = alone.solve(b, xa, rtol=1e-10, maxit=100)
        assert abs(ia.iterations - inf.iterations) <= 1
        assert np.linalg.norm(host(xa) - host(x)) <= 1e-9 * np.linalg.norm(host(xa))


def test_batch_initial_guess_and_repeat():
    import torch
    shapes = [(2, 4, 2), (2, 3, 5), (3, 2, 3)]
    bt = SIPGBatch(_params(shapes, SIPG_FP32))
    bs = _rhs(bt, 320)
    xs = [torch.zeros_like(b) for b in bs]
    first = bt.solve(bs, xs, rtol=1e-10)
    # restarting from the converged solutions takes no iteration
    again = bt.solve(bs, xs, rtol=1e-10)
    assert all(i.iterations == 0 and i.status == 0 for i in again)
    # the same solve twice gives the same bits (deterministic reductions)
    ys = [torch.zeros_like(b) for b in bs]
    second = bt.solve(bs, ys, rtol=1e-10)
    zs = [torch.zeros_like(b) for b in bs]
    bt.solve(bs, zs, rtol=1e-10)
    for a, b_, i1, i2 in zip(ys, zs, first, second):
        assert torch.equal(a, b_) and i1.iterations == i2.iterations


def test_batch_rejects_aliased_member_vectors():
    import torch
    bt = SIPGBatch(_params([(2, 3, 2), (2, 4, 2)], SIPG_FP64))
    bs = _rhs(bt, 330)
    xs = [torch.zeros_like(bs[0]), bs[1]]
    with pytest.raises(SipgError, match="member 1"):
        bt.solve(bs, xs)


@pytest.fixture(scope="module")
def ragged64():
    shapes = [(2, L, k) for L, k in inputs.ragged_problems(4)]
    return shapes, SIPGBatch(_params(shapes, SIPG_FP32))


def test_ragged64_full_batch(ragged64):
    import torch
    shapes, bt = ragged64
    assert len(bt) == 64
    bs = _rhs(bt, 1000)
    xs = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, rtol=1e-10, maxit=100)
    assert all(i.status == 0 and i.rel_residual <= 1e-10 for i in infos)
    # exact solves for the largest members and a seeded sample of the rest
    order = sorted(range(64), key=lambda i: -bt.members[i].ndofs())
    rng = np.random.default_rng(5)
    pick = sorted(set(order[:3]) | set(int(i) for i in rng.choice(64, size=6, replace=False)))
    for i in pick:
        d, L, k = shapes[i]
        u = GlobalFD(d, k, 1 << L).solve(host(bs[i]))
        err = np.linalg.norm(host(xs[i]) - u) / np.linalg.norm(u)
        assert err < 1e-8, (i, L, k, err)


FUSED = [(2, 3, 2), (2, 5, 6), (2, 4, 3), (2, 6, 2), (2, 2, 5), (2, 5, 4), (2, 3, 6), (2, 4, 4)]


@pytest.mark.parametrize("rtol", [1e-10, 1e-12])
def test_fused_batch_matches_direct_and_per_member_path(monkeypatch, rtol):
    import torch
    monkeypatch.setenv("SIPG_BATCH_FUSED", "1")
    bt = SIPGBatch(_params(FUSED, SIPG_FP32))
    bs = _rhs(bt, 340)
    xs = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, rtol=rtol, maxit=100)
    monkeypatch.setenv("SIPG_BATCH_FUSED", "0")
    ref = SIPGBatch(_params(FUSED, SIPG_FP32))
    ys = [torch.zeros_like(b) for b in bs]
    rinfos = ref.solve(bs, ys, rtol=rtol, maxit=100)
    for (d, L, k), b, x, y, inf, rinf in zip(FUSED, bs, xs, ys, infos, rinfos):
        assert inf.status == 0 and inf.rel_residual <= rtol
        u = GlobalFD(d, k, 1 << L).solve(host(b))
        err = np.linalg.norm(host(x) - u) / np.linalg.norm(u)
        assert err < (1e-8 if rtol >= 1e-10 else 1e-9), (L, k, err)
        # the same preconditioner (FP32 colour passes of the same
        # arithmetic), so the same iterations and nearly the same iterates
        assert abs(inf.iterations - rinf.iterations) <= 1
        assert np.linalg.norm(host(x) - host(y)) <= 1e-8 * np.linalg.norm(host(y))


def test_fused_batch_repeat_is_deterministic(monkeypatch):
    import torch
    monkeypatch.setenv("SIPG_BATCH_FUSED", "1")
    bt = SIPGBatch(_params(FUSED, SIPG_FP32))
    bs = _rhs(bt, 350)
    xs = [torch.zeros_like(b) for b in bs]
    first = bt.solve(bs, xs, rtol=1e-10)
    ys = [torch.zeros_like(b) for b in bs]
    second = bt.solve(bs, ys, rtol=1e-10)
    for a, b_, i1, i2 in zip(xs, ys, first, second):
        assert torch.equal(a, b_) and i1.iterations == i2.iterations
    # from the converged solutions: no iteration
    again = bt.solve(bs, xs, rtol=1e-10)
    assert all(i.iterations == 0 and i.status == 0 for i in again)


def test_fused_ragged64_matches_per_member_path(monkeypatch, ragged64):
    import torch
    shapes, ref = ragged64
    monkeypatch.setenv("SIPG_BATCH_FUSED", "1")
    bt = SIPGBatch(_params(shapes, SIPG_FP32))
    bs = _rhs(bt, 1100)
    xs = [torch.zeros_like(b) for b in bs]
    ys = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, rtol=1e-10, maxit=100)
    rinfos = ref.solve(bs, ys, rtol=1e-10, maxit=100)
    for x, y, i, r in zip(xs, ys, infos, rinfos):
        assert i.status == 0 and i.rel_residual <= 1e-10
        assert abs(i.iterations - r.iterations) <= 1
        assert np.linalg.norm(host(x) - host(y)) <= 1e-8 * np.linalg.norm(host(y))
