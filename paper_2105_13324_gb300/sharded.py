"""One acquisition split over several GPUs (one process per GPU).

Transport: rank g runs histories [g H / G, (g + 1) H / G).  Histories are
independent (paper Sec. 2), so the counts of the ranges add up exactly to
those of the whole acquisition.

Matrix: the views are cut into G contiguous blocks, part p holding views
[p V / G, (p + 1) V / G).  Each rank routes its tally events to the rank that
owns their view (one all-to-all of event keys) and assembles the rows of its
views from every range: its part of the count matrix C of Eq. (IMC), bit for
bit, with n_v counted over the whole range [0, H).

ML-EM (Eq. (MLEM), Sec. 5.1): the forward projection and the ratio y / (A x)
involve only a rank's own rows; the back-projection sum_j A_jv r_j runs over
all rows, so each rank's partial N-vector is summed by one all-reduce per
iteration, after which the multiplicative update is the same on every rank.
The sensitivity s_v = sum_j A_jv and sum_j y_j are all-reduced once.

The arithmetic runs in the library (``LibraryOps``); ``TorchComm`` moves data
with torch.distributed (NCCL between GPUs; gloo with CPU tensors).  Both are
passed in, so the same partitioning, exchange and iteration run everywhere.
"""
from __future__ import annotations


def history_range(rank: int, world: int, n_histories: int):
    """(first, count) of rank's share of histories 0 .. n_histories-1."""
    first = rank * n_histories // world
    return first, (rank + 1) * n_histories // world - first


def view_block(part: int, n_parts: int, n_views: int):
    """Views [v0, v1) owned by part `part` of `n_parts`."""
    return part * n_views // n_parts, (part + 1) * n_views // n_parts


class TorchComm:
    """torch.distributed collectives on tensors of the process group's
    device (CUDA tensors with NCCL, CPU tensors with gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def all_to_all(self, t, send_counts):
        """Send send_counts[p] consecutive elements of t to rank p (in rank
        order); returns what every rank sent here, concatenated in rank
        order."""
        import torch
        sc = torch.tensor(send_counts, dtype=torch.int64, device=t.device)
        rc = torch.empty_like(sc)
        self.dist.all_to_all_single(rc, sc, group=self.group)
        recv_counts = [int(c) for c in rc.cpu()]
        out = torch.empty(sum(recv_counts), dtype=t.dtype, device=t.device)
        self.dist.all_to_all_single(out, t, recv_counts, [int(c) for c in send_counts], group=self.group)
        return out

    def all_reduce_(self, t):
        """In-place sum over ranks."""
        self.dist.all_reduce(t, group=self.group)
        return t


class LibraryOps:
    """The split's arithmetic, all of it in libmcspect (CUDA tensors)."""

    def __init__(self, mc):
        self.mc = mc

    def tally(self, plan, first, count, seed):
        keys, _ = self.mc.mc_plan_tally(plan, first, count, seed)
        return keys

    def route(self, keys, n_rows, rows_per_view, n_parts):
        return self.mc.mc_events_route(keys, n_rows, rows_per_view, n_parts)

    def assemble(self, keys, n_rows, n_cols, first, count):
        return self.mc.mc_system_from_keys(n_rows, n_cols, keys, first, count)

    def sensitivity(self, system, n_cols):
        import torch
        s = torch.empty(n_cols, dtype=torch.float64, device="cuda")
        return self.mc.mc_sensitivity(system, s)

    def vector_sum(self, v):
        import torch
        return self.mc.mc_vector_sum(v, torch.empty(1, dtype=torch.float64, device="cuda"))

    def start(self, sens, sum_y, n_cols):
        import torch
        return self.mc.mc_mlem_start(sens, sum_y, torch.empty(n_cols, dtype=torch.float32, device="cuda"))

    def vector(self, n):
        import torch
        return torch.empty(n, dtype=torch.float32, device="cuda")

    def project_ratio(self, system, x, y, r):
        self.mc.mc_project_ratio(system, x, y, r)

    def backproject(self, system, r, b):
        self.mc.mc_backproject(system, r, b)

    def em_update(self, sens, b, x):
        # x <- x b / s (0 where s = 0): one preconditioned step of unit length
        self.mc.mc_pgd_step(1.0, sens, b, x)


def split_build(ops, comm, plan, n_rows: int, n_cols: int, rows_per_view: int, n_histories: int, seed: int):
    """This rank's part of the matrix of histories 0 .. n_histories-1: the
    rows of its views (renumbered from 0), with n_v over all histories.
    Returns (system, (v0, v1)) with [v0, v1) the rank's views."""
    first, count = history_range(comm.rank, comm.world, n_histories)
    keys = ops.tally(plan, first, count, seed)
    routed, counts = ops.route(keys, n_rows, rows_per_view, comm.world)
    mine = comm.all_to_all(routed, counts)
    v0, v1 = view_block(comm.rank, comm.world, n_rows // rows_per_view)
    return ops.assemble(mine, (v1 - v0) * rows_per_view, n_cols, 0, n_histories), (v0, v1)


def split_mlem(ops, comm, system, y_part, n_rows_part: int, n_cols: int, n_iter: int):
    """n_iter ML-EM updates from the uniform start image, over a matrix whose
    rows are split across the ranks; y_part holds this rank's rows.  Returns
    the image (the same on every rank)."""
    sens = comm.all_reduce_(ops.sensitivity(system, n_cols))
    sum_y = float(comm.all_reduce_(ops.vector_sum(y_part))[0])
    x = ops.start(sens, sum_y, n_cols)
    r = ops.vector(n_rows_part)
    b = ops.vector(n_cols)
    for _ in range(n_iter):
        ops.project_ratio(system, x, y_part, r)
        ops.backproject(system, r, b)
        comm.all_reduce_(b)
        ops.em_update(sens, b, x)
    return x
