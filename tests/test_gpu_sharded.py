"""The split of one acquisition (paper_2105_13324_gb300.sharded) with the
library's kernels on one GPU, through the C ABI.

G virtual ranks run as threads of one process on the same GPU; their
all-to-all and all-reduce are emulated in-process (rank order, on the
device), so the library's tally, routing, assembly and ML-EM pieces run
exactly as they would with one GPU per rank.  Pinned against the oracle: in
FP64 verification mode every part equals the rows of its views of the
oracle's count matrix exactly, and the split ML-EM image equals oracle.mlem
on that matrix; in FP32 every part equals the rows of the whole-range build
and the image the single-system mlem_iterate image.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

N_ITER = 10


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


class _Shared:
    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world, timeout=300)
        self.slots = [None] * world


class ThreadComm:
    """all_to_all / all_reduce among threads (virtual ranks) of one process."""

    def __init__(self, shared, rank):
        self.sh, self.rank, self.world = shared, rank, shared.world

    def all_to_all(self, t, send_counts):
        import torch
        self.sh.slots[self.rank] = (t, list(send_counts))
        self.sh.barrier.wait()
        pieces = []
        for src in range(self.world):
            ts, cs = self.sh.slots[src]
            off = sum(cs[:self.rank])
            pieces.append(ts[off:off + cs[self.rank]])
        out = torch.cat(pieces)
        self.sh.barrier.wait()
        return out

    def all_reduce_(self, t):
        torch_sync()
        self.sh.slots[self.rank] = t.clone()
        self.sh.barrier.wait()
        total = self.sh.slots[0].clone()
        for src in range(1, self.world):
            total += self.sh.slots[src]
        self.sh.barrier.wait()
        t.copy_(total)
        torch_sync()
        return t


def torch_sync():
    import torch
    torch.cuda.synchronize()


def _run_split(mc, w, precision, H, y, world):
    from paper_2105_13324_gb300 import sharded
    plan = mc.Plan(w.phantom, w.geometry, precision)
    rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
    M = w.geometry.n_views * rpv
    N = int(np.prod(w.phantom.shape))
    sh = _Shared(world)
    results, errors = [None] * world, []

    def rank_main(rank):
        import torch
        try:
            comm = ThreadComm(sh, rank)
            ops = sharded.LibraryOps(mc)
            sysm, (v0, v1) = sharded.split_build(ops, comm, plan, M, N, rpv, H, w.seed)
            y_part = torch.as_tensor(np.ascontiguousarray(y[v0 * rpv:v1 * rpv])).cuda()
            x = sharded.split_mlem(ops, comm, sysm, y_part, (v1 - v0) * rpv, N, N_ITER)
            torch.cuda.synchronize()
            results[rank] = ((v0, v1), sysm.export_csc(), x.cpu().numpy().astype(np.float64))
            sysm.free()
        except Exception as e:        # reported by the main thread
            errors.append(e)
            sh.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    plan.free()
    if errors:
        raise errors[0]
    return results, rpv


def test_split_fp64_equals_the_oracle(mc):
    w = P.workload("water32")
    pr = oracle.Problem(w.phantom, w.geometry)
    H = 1_000_000
    _, c_all, nv, _ = oracle.build_system(pr, w.seed, H)
    c_all = c_all.tocsr()
    a_all = oracle.system_matrix(c_all, nv)
    y = P.poisson_counts(a_all @ w.phantom.activity.ravel().astype(np.float64), 1e5, 3)
    want = oracle.mlem(a_all, y, oracle.mlem_init(a_all, y), N_ITER)
    results, rpv = _run_split(mc, w, "fp64", H, y, world=3)
    views = []
    for (v0, v1), (cp, ri, cnt, n_v), x in results:
        views.extend(range(v0, v1))
        part = c_all[v0 * rpv:v1 * rpv].tocsc()
        part.sort_indices()
        np.testing.assert_array_equal(cp, part.indptr)
        np.testing.assert_array_equal(ri, part.indices)
        np.testing.assert_array_equal(cnt, part.data)
        np.testing.assert_array_equal(n_v, nv)
        assert np.linalg.norm(x - want) / np.linalg.norm(want) <= 1e-5
    assert views == list(range(w.geometry.n_views))


def test_split_fp32_equals_the_whole_build(mc):
    import torch
    w = P.workload("torso64")
    H = 8_000_000
    plan = mc.Plan(w.phantom, w.geometry, "fp32")
    whole = plan.build(0, H, w.seed)
    cp_all, ri_all, cnt_all, _ = whole.export_csc()
    act = torch.as_tensor(w.phantom.activity.ravel()).cuda()
    q = torch.zeros(whole.shape[0], device="cuda")
    mc.mc_project(whole, act, q)
    y = P.poisson_counts(q.cpu().numpy(), 1e6, 4)
    x1 = torch.zeros(whole.shape[1], device="cuda")
    yd = torch.as_tensor(y).cuda()
    mc.mc_mlem_init(whole, yd, x1)
    mc.mlem_iterate(whole, yd, x1, N_ITER)
    x1 = x1.cpu().numpy().astype(np.float64)
    import scipy.sparse as sp
    c_all = sp.csc_matrix((cnt_all, ri_all, cp_all), shape=whole.shape).tocsr()
    whole.free()
    plan.free()
    results, rpv = _run_split(mc, w, "fp32", H, y, world=4)
    for (v0, v1), (cp, ri, cnt, _), x in results:
        part = c_all[v0 * rpv:v1 * rpv].tocsc()
        part.sort_indices()
        np.testing.assert_array_equal(cp, part.indptr)
        np.testing.assert_array_equal(ri, part.indices)
        np.testing.assert_array_equal(cnt, part.data)
        assert np.linalg.norm(x - x1) / np.linalg.norm(x1) <= 1e-6
