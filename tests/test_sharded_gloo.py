"""The split of one acquisition over ranks (paper_2105_13324_gb300.sharded),
run as 2 and 3 gloo ranks on the CPU.

The partitioning, the event exchange (all-to-all), the all-reduces and the
ML-EM loop are the product's own code; the arithmetic it calls is supplied
by an oracle-backed stand-in for the library (float64, CPU tensors), so the
test needs no GPU.  Pinned against the single-process oracle: every rank's
part equals the rows of its views of the whole count matrix exactly
(histories are independent, Sec. 2: counts of disjoint ranges add), and the
split ML-EM image equals oracle.mlem on the whole matrix (Eq. (MLEM): the
back-projection sums over detector bins, so bins split by views).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2105_13324_gb300 import phantoms as P

H = 600_000
N_ITER = 8


class OracleOps:
    """The arithmetic of the split, from the oracle (float64, CPU)."""

    def tally(self, prob, first, count, seed):
        rows, cols, _ = oracle.run(prob, seed, first, count, threads=2)
        return torch.as_tensor(cols.astype(np.int64) * prob.n_rows + rows.astype(np.int64))

    def route(self, keys, n_rows, rows_per_view, n_parts):
        k = keys.numpy()
        j, v = k % n_rows, k // n_rows
        n_views = n_rows // rows_per_view
        view = j // rows_per_view
        owner = np.zeros(n_views, np.int64)
        bounds = [p * n_views // n_parts for p in range(n_parts + 1)]
        for p in range(n_parts):
            owner[bounds[p]:bounds[p + 1]] = p
        out, counts = [], []
        for p in range(n_parts):
            sel = owner[view] == p
            m_p = (bounds[p + 1] - bounds[p]) * rows_per_view
            out.append(v[sel] * m_p + (j[sel] - bounds[p] * rows_per_view))
            counts.append(int(sel.sum()))
        return torch.as_tensor(np.concatenate(out)), counts

    def assemble(self, keys, n_rows, n_cols, first, count):
        k = keys.numpy()
        c = oracle.system_counts(k % n_rows, k // n_rows, n_rows, n_cols)
        return c, oracle.system_matrix(c, oracle.histories_per_voxel(n_cols, first, count))

    def sensitivity(self, system, n_cols):
        return torch.as_tensor(oracle.sensitivity(system[1]))

    def vector_sum(self, v):
        return torch.tensor([float(np.sum(v.numpy().astype(np.float64)))], dtype=torch.float64)

    def start(self, sens, sum_y, n_cols):
        s = sens.numpy()
        return torch.as_tensor(np.where(s > 0, sum_y / s.sum(), 0.0))

    def vector(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def project_ratio(self, system, x, y, r):
        q = system[1] @ x.numpy()
        out = np.zeros_like(q)
        np.divide(y.numpy().astype(np.float64), q, out=out, where=q > 0)
        r.copy_(torch.as_tensor(out))

    def backproject(self, system, r, b):
        b.copy_(torch.as_tensor(system[1].T @ r.numpy()))

    def em_update(self, sens, b, x):
        s = sens.numpy()
        out = np.zeros_like(s)
        np.divide(x.numpy() * b.numpy(), s, out=out, where=s > 0)
        x.copy_(torch.as_tensor(out))


def _problem():
    w = P.workload("water32")
    return w, oracle.Problem(w.phantom, w.geometry)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2105_13324_gb300 import sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, pr = _problem()
        rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
        comm = sharded.TorchComm()
        ops = OracleOps()
        (c, a), (v0, v1) = sharded.split_build(ops, comm, pr, pr.n_rows, pr.n_voxels, rpv, H, w.seed)
        y = np.load(os.path.join(out_dir, "y.npy"))
        y_part = torch.as_tensor(y[v0 * rpv:v1 * rpv])
        x = sharded.split_mlem(ops, comm, (c, a), y_part, (v1 - v0) * rpv, pr.n_voxels, N_ITER)
        c = c.tocsc()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), views=np.array([v0, v1]), indptr=c.indptr,
                 indices=c.indices, data=c.data, x=x.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_split_build_and_mlem_on_gloo_ranks_equal_the_whole(tmp_path, world):
    w, pr = _problem()
    rows, cols, _ = oracle.run(pr, w.seed, 0, H)
    c_all = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels).tocsr()
    a_all = oracle.system_matrix(c_all, oracle.histories_per_voxel(pr.n_voxels, 0, H))
    y = P.poisson_counts(a_all @ w.phantom.activity.ravel().astype(np.float64), 1e5, 3)
    np.save(tmp_path / "y.npy", y)
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    want = oracle.mlem(a_all, y, oracle.mlem_init(a_all, y), N_ITER)
    rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
    covered = []
    for rank in range(world):
        d = np.load(tmp_path / f"rank{rank}.npz")
        v0, v1 = (int(v) for v in d["views"])
        covered.extend(range(v0, v1))
        part = c_all[v0 * rpv:v1 * rpv].tocsc()
        part.sort_indices()
        np.testing.assert_array_equal(d["indptr"], part.indptr)
        np.testing.assert_array_equal(d["indices"], part.indices)
        np.testing.assert_array_equal(d["data"], part.data)
        np.testing.assert_allclose(d["x"], want, rtol=1e-12, atol=1e-14 * want.max())
    assert covered == list(range(w.geometry.n_views))   # every view owned once, in order
