"""Multi-GPU host logic on CPU: the object partition (longest-processing-time
first) and the two-rank flow of a sharded step over gloo (each rank derives
the same partition, trains only its own objects, and the step time is the
maximum over ranks).  No GPU is involved."""

import itertools
import os
import socket

import numpy as np
import pytest

from paper_2503_01582_gb300.shard import lpt_partition, makespan, object_cost, rank_objects

# (log2T, W, H) of the category table that the 32-object workload draws from
CATEGORIES = [(17, 32, 1), (16, 32, 2), (19, 64, 3), (18, 64, 2), (14, 16, 1), (17, 32, 2), (14, 16, 1),
              (15, 16, 2), (19, 64, 3)]


def _table_costs(orc, n_objects=32, seed=7):
    rng = np.random.default_rng(seed)
    costs = []
    for i in range(n_objects):
        log2T, W, H = CATEGORIES[i % len(CATEGORIES)]
        a = orc.Arch(L=16, F=2, log2T=log2T, n_min=16, n_max=2048, width=W, hidden=H)
        rays = 32 * int(round(8 * 2 ** (5 * rng.random())))
        costs.append(object_cost(16, 2, W, H, orc.param_count(a), rays * 48, feature_bytes=2))
    return costs


def _optimum(costs, world):
    best = float("inf")
    for assign in itertools.product(range(world), repeat=len(costs)):
        loads = [0.0] * world
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


def test_lpt_covers_disjoint_and_within_graham_bound():
    rng = np.random.default_rng(0)
    for trial in range(60):
        n = int(rng.integers(1, 9))
        world = int(rng.integers(1, 4))
        costs = list(rng.integers(1, 100, n).astype(float))
        parts = lpt_partition(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(n))
        opt = _optimum(costs, world)
        assert makespan(costs, parts) <= (4 / 3 - 1 / (3 * world)) * opt + 1e-9


def test_lpt_known_cases():
    # Graham's tight example for two machines: 3, 3, 2, 2, 2 -> LPT 7, optimum 6
    parts = lpt_partition([3, 3, 2, 2, 2], 2)
    assert makespan([3, 3, 2, 2, 2], parts) == 7
    assert lpt_partition([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]
    assert lpt_partition([], 3) == [[], [], []]
    assert lpt_partition([1.0, 1.0], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        lpt_partition([1.0], 0)
    with pytest.raises(ValueError):
        rank_objects([1.0], 2, 2)


def test_object_cost_terms():
    # 1 sample, L=F=1, W=1, H=1: gather+scatter 8*(4+4) = 64, MLP 2*(1 + 0 + 4) = 10
    assert object_cost(1, 1, 1, 1, 0, 1) == 74.0
    assert object_cost(1, 1, 1, 1, 10, 0) == 280.0
    # FP16 features read 2 bytes instead of 4
    assert object_cost(16, 2, 64, 2, 0, 1, feature_bytes=2) == 8 * 32 * 6 + 2 * (64 * 32 + 64 * 64 + 256)


def test_table_partition_is_balanced(orc):
    costs = _table_costs(orc)
    for world in (2, 4, 8):
        parts = lpt_partition(costs, world)
        # the makespan is within 4/3 of the average load (a lower bound of the optimum),
        # or equals the largest single object when that object dominates
        lower = max(sum(costs) / world, max(costs))
        assert makespan(costs, parts) <= (4 / 3) * lower + 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out_dir):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = rank_objects(costs, world, rank)
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    # stand-in for the timed step: this rank's load (the step time of its shard)
    t = torch.tensor([sum(costs[i] for i in mine)], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr((mine, everyone, float(t.item()))))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_partition_and_time(orc, tmp_path):
    import torch.multiprocessing as mp

    costs = _table_costs(orc)
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), costs, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    parts = lpt_partition(costs, world)
    for r, (mine, everyone, tmax) in enumerate(res):
        assert mine == parts[r]
        assert everyone == parts  # every rank derived the same partition
        assert tmax == pytest.approx(makespan(costs, parts))
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))


# ------------------------------------------------------- multi-GPU Reptile meta step (host flow)
class _HostCtx:
    """Stands in for a Context on the CPU: parameters are float64 numpy arrays and
    the inner "training" moves each task by a fixed per-task offset, so the meta
    step's flow (begin, inner steps, task sum, all-reduce, apply) runs over gloo."""

    def __init__(self, n_params, theta0):
        self.theta = {0: np.array(theta0, np.float64)}
        self.n = n_params

    def param_count(self, obj):
        return self.n

    def reptile_begin(self, meta, tasks):
        for t in tasks:
            self.theta[t] = self.theta[meta].copy()

    def train_step(self, batches, opts, loss=None):
        for b in batches:
            self.theta[b["obj"]] += b["delta"]

    def reptile_update(self, meta, tasks, beta):
        import oracle

        oracle.reptile(self.theta[meta], [self.theta[t] for t in tasks], beta)

    def reptile_task_sum(self, tasks, out):
        import torch

        out.copy_(torch.from_numpy(np.sum([self.theta[t] for t in tasks], axis=0)))

    def reptile_apply(self, meta, task_sum, n_total, beta):
        import oracle

        mean = task_sum.numpy().astype(np.float64) / n_total
        oracle.reptile(self.theta[meta], [mean], beta)

    def sync(self):
        pass


def _meta_worker(rank, world, port, n_tasks, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2503_01582_gb300.meta import meta_step, split_tasks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    theta0 = rng.normal(size=64)
    deltas = rng.normal(size=(n_tasks, 64))
    mine = split_tasks(n_tasks, world, rank)
    ctx = _HostCtx(64, theta0)
    ids = [1 + t for t in mine]
    inner = [[dict(obj=1 + t, delta=deltas[t] / 3) for t in mine] for _ in range(3)]
    n_total = meta_step(ctx, 0, ids, inner, None, 0.25, group=dist.group.WORLD,
                        task_sum=torch.zeros(64, dtype=torch.float64))
    np.save(os.path.join(out_dir, f"meta{rank}.npy"), ctx.theta[0])
    with open(os.path.join(out_dir, f"n{rank}.txt"), "w") as f:
        f.write(str(n_total))
    dist.destroy_process_group()


def test_split_tasks_covers_evenly():
    from paper_2503_01582_gb300.meta import split_tasks

    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            parts = [split_tasks(n, world, r) for r in range(world)]
            assert sorted(i for p in parts for i in p) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_two_gloo_ranks_meta_step_equals_single_process(orc, tmp_path):
    """Tasks split over two ranks, sums all-reduced, outer update applied on each
    rank: every rank ends with the meta-parameters of the whole meta-batch
    updated at once (Eq. 2 over all 5 tasks)."""
    import torch.multiprocessing as mp

    n_tasks = 5
    mp.start_processes(_meta_worker, args=(2, _free_port(), n_tasks, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    rng = np.random.default_rng(0)
    theta0 = rng.normal(size=64)
    deltas = rng.normal(size=(n_tasks, 64))
    want = theta0.copy()
    orc.reptile(want, [theta0 + d for d in deltas], 0.25)
    for r in range(2):
        assert open(tmp_path / f"n{r}.txt").read() == str(n_tasks)
        np.testing.assert_allclose(np.load(tmp_path / f"meta{r}.npy"), want, rtol=0, atol=1e-12)
