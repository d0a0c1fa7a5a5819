"""GPU parity of the batched API over uneven problems (the batched configuration).

Every problem's right-hand sides are compared with the oracle's normal-equation solve
of that problem: ||x - x*|| / ||x*|| <= 1e-10 for each of the 8 right-hand sides.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import colmajor, relerr, to_np_colmajor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ils():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2203_15340_gb300 as pkg
    return pkg


def run_batch(ils, insts, opts, tol=1e-12):
    import torch
    Ats = [colmajor(inst.A) for inst in insts]
    bs = ils.BatchSolver(Ats, [inst.p for inst in insts], opts)
    k = insts[0].b.shape[1]
    Bts = [colmajor(inst.b) for inst in insts]
    Xts = [torch.zeros((k, inst.n), dtype=torch.float64, device="cuda") for inst in insts]
    infos = bs.solve(Bts, Xts, tol=tol)
    torch.cuda.synchronize()
    out = [to_np_colmajor(X) for X in Xts]
    bs.close()
    return out, infos


@pytest.mark.parametrize("precision", [0, 2])
def test_batched_subset_uneven(ils, precision):
    idx = [0, 5, 17, 42, 77, 101, 150, 201, 255]
    insts = W.config4_batched(indices=idx)
    opts = ils.options(precision=precision)
    X, infos = run_batch(ils, insts, opts)
    for inst, x, info in zip(insts, X, infos):
        assert info.status == ils.ILS_OK
        xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
        for j in range(inst.b.shape[1]):
            assert relerr(x[:, j], xs[:, j]) <= 1e-10, (inst.name, j)


def test_batched_matches_single_handles(ils):
    import torch
    insts = W.config4_batched(indices=[3, 9], k=3)
    X, _ = run_batch(ils, insts, ils.options())
    for inst, xb in zip(insts, X):
        s = ils.Solver(colmajor(inst.A), inst.p)
        Xs = torch.zeros((3, inst.n), dtype=torch.float64, device="cuda")
        s.solve_many(colmajor(inst.b), Xs, tol=1e-12)
        assert np.array_equal(to_np_colmajor(Xs), xb)  # same kernels, same order: bitwise equal
        s.close()


def test_batched_full_config(ils):
    """All 256 problems of the batched configuration, 8 right-hand sides each, BF16 sweeps."""
    insts = W.config4_batched()
    X, infos = run_batch(ils, insts, ils.options(precision=2))
    worst = 0.0
    for inst, x, info in zip(insts, X, infos):
        assert info.status == ils.ILS_OK
        xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
        worst = max(worst, max(relerr(x[:, j], xs[:, j]) for j in range(8)))
    assert worst <= 1e-10


def test_batched_rejects_non_spd_member(ils):
    good = W.dense_gaussian(80, 10, 8, 0.2, 1, k=2)
    bad = W.dense_gaussian(60, 40, 10, 3.0, 2, k=2)
    with pytest.raises(ils.ILSError) as e:
        ils.BatchSolver([colmajor(good.A), colmajor(bad.A)], [good.p, bad.p])
    assert e.value.code == ils.ILS_ERR_NOT_SPD


def _graph_case(ils, insts, opts, steps, refactor=False):
    import torch
    s = torch.cuda.Stream()
    Ats = [colmajor(inst.A) for inst in insts]
    k = insts[0].b.shape[1]
    Bts = [colmajor(inst.b) for inst in insts]
    X_host = [torch.zeros((k, inst.n), dtype=torch.float64, device="cuda") for inst in insts]
    X_graph = [torch.zeros((k, inst.n), dtype=torch.float64, device="cuda") for inst in insts]
    with torch.cuda.stream(s):
        bs = ils.BatchSolver(Ats, [inst.p for inst in insts], opts, stream=s)
        bs.solve(Bts, X_host, tol=1e-12, stream=s)
        bs.capture(Bts, X_graph, refactor=refactor, steps=steps, tol=1e-12, stream=s)
        infos = bs.run(stream=s)
    torch.cuda.synchronize()
    return bs, s, Ats, Bts, X_host, X_graph, infos


@pytest.mark.parametrize("steps", [8, 1])
def test_batched_graph_replay_matches_host_driven(ils, steps):
    """One graph launch replays the batch solve; with too few captured steps the host-driven
    path finishes it.  Same kernels in the same order: bitwise equal to ils_batch_solve."""
    insts = W.config4_batched(indices=[3, 9, 17, 40], k=3)
    bs, s, _, _, X_host, X_graph, infos = _graph_case(ils, insts, ils.options(precision=2), steps)
    for xh, xg, info in zip(X_host, X_graph, infos):
        assert info.status == ils.ILS_OK
        assert np.array_equal(to_np_colmajor(xh), to_np_colmajor(xg))
    bs.close()


def test_batched_graph_refactor_reads_new_values(ils):
    """A captured refactor re-reads A: doubling every A halves every solution."""
    import torch
    insts = W.config4_batched(indices=[5, 12], k=2)
    bs, s, Ats, _, _, X_graph, _ = _graph_case(ils, insts, ils.options(precision=1), 8, refactor=True)
    with torch.cuda.stream(s):
        for At in Ats:
            At.mul_(2.0)
        infos = bs.run(stream=s)
    torch.cuda.synchronize()
    for inst, X, info in zip(insts, X_graph, infos):
        assert info.status == ils.ILS_OK
        xs = O.normal_equation_solve(2.0 * inst.A, inst.b, inst.p)
        x = to_np_colmajor(X)
        for j in range(x.shape[1]):
            assert relerr(x[:, j], xs[:, j]) <= 1e-10
    bs.close()


def test_batched_graph_full_config(ils):
    """All 256 problems, 8 right-hand sides each, BF16 sweeps, setup and solve in one graph."""
    import torch
    insts = W.config4_batched()
    bs, s, _, _, _, X_graph, infos = _graph_case(ils, insts, ils.options(precision=2), 8, refactor=True)
    worst = 0.0
    for i in range(0, len(insts), 8):
        inst, info = insts[i], infos[i]
        assert info.status == ils.ILS_OK
        xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
        x = to_np_colmajor(X_graph[i])
        worst = max(worst, max(relerr(x[:, j], xs[:, j]) for j in range(8)))
    assert worst <= 1e-10
    bs.close()


def test_batched_graph_repeated_replays_are_identical(ils):
    """Replays of one captured setup+solve give the same statuses and bitwise the same X every
    time, with all 256 problems' kernels in flight together (a race between CTAs of one
    launch would show up here as a spurious status or a changed answer)."""
    import torch
    insts = W.config4_batched()
    bs, s, _, _, _, X_graph, infos = _graph_case(ils, insts, ils.options(precision=2), 8, refactor=True)
    first = [to_np_colmajor(X) for X in X_graph]
    for rep in range(4):
        with torch.cuda.stream(s):
            infos = bs.run(stream=s)
        torch.cuda.synchronize()
        assert all(info.status == ils.ILS_OK for info in infos), rep
        for x0, X in zip(first, X_graph):
            assert np.array_equal(x0, to_np_colmajor(X)), rep
    bs.close()
