"""Block sharding (the multi-GPU decomposition) on one GPU, shard after shard.

Every unordered k-point block {k, q} belongs to one shard; a sharded plan
computes the partial V_x c and E_x of its blocks.  The shards' partial results
must add up to the unsharded result, with the pair symmetry on (shared grids,
the accumulators of every k-point at once) and off, and the shards' transforms
must add up to the unsharded count.
"""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def rhombo24():
    return synth.make_workload("rhombo24", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                               synth.monkhorst_pack(2), 2.4, 4, 6, [1.0, 1.0, 0.75, 0.3], 21)


def run_shard(xx, wl, prec, shard, n, sym=True):
    plan = xx.Plan.from_workload(wl, precision=prec)
    plan.set_batch(3, 3)
    plan.set_pair_symmetry(sym)
    plan.set_shard(shard, n)
    c = gu.dev(wl.c_tgt)
    ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy(), float(ex[0].item()), plan.info()["pairs_transformed"]
    plan.close()
    return out


@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("n", [2, 3, 8])
def test_shards_sum_to_the_unsharded_operator(gpu, sym, n):
    torch, xx = gpu
    wl = rhombo24()
    full, e_full, t_full = run_shard(xx, wl, 1, 0, 1, sym)
    parts = [run_shard(xx, wl, 1, r, n, sym) for r in range(n)]
    vx = sum(p[0] for p in parts)
    e = 0.0
    for p in parts:          # shares added in shard order
        e += p[1]
    assert gu.rel_max(vx, full) <= 1e-12
    assert abs(e - e_full) <= 1e-12 * abs(e_full)
    assert sum(p[2] for p in parts) == t_full
    owner = xx.xx_shard_blocks(wl.nk, wl.n_occ, wl.n_tgt, n)
    for r, p in enumerate(parts):
        if not np.any(owner == r):
            assert p[2] == 0 and float(np.abs(p[0]).max()) == 0.0


def test_sharded_plan_refuses_unsharded_derivatives(gpu):
    torch, xx = gpu
    wl = rhombo24()
    plan = xx.Plan.from_workload(wl, precision=1)
    plan.set_shard(1, 2)
    c, w = gu.dev(wl.c_tgt), gu.dev(wl.w_tgt)
    with pytest.raises(xx.XXError):
        plan.backward(c, w, grad_ex=1.0)          # dE/dmu is not sharded
    with pytest.raises(xx.XXError):
        plan.strain_derivative(c, w)
    with pytest.raises(xx.XXError):
        plan.set_shard(2, 2)
    plan.close()


@pytest.mark.parametrize("n", [1, 2, 8])
@pytest.mark.parametrize("batch", [(3, 3), None])
def test_bench_schedule_model_matches_sharded_plans(gpu, n, batch):
    """bench.py checks its launch-schedule model against each rank's transform count;
    the model with the library's block assignment must give every shard's count, with
    one q-point per batch and with the default multi-q batches."""
    torch, xx = gpu
    import bench
    wl = rhombo24()
    owner = xx.xx_shard_blocks(wl.nk, wl.n_occ, wl.n_tgt, n)
    for r in range(n):
        plan = xx.Plan.from_workload(wl, precision=0)
        if batch:
            plan.set_batch(*batch)
        plan.set_shard(r, n)
        c = gu.dev(wl.c_tgt)
        plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        info = plan.info()
        plan.close()

        def owned(k, q, r=r):
            k, q = min(k, q), max(k, q)
            return owner[k * wl.nk - k * (k - 1) // 2 + (q - k)] == r
        sched = bench.batch_schedule(wl.nk, wl.n_occ, wl.n_tgt, info["targets_per_batch"],
                                     info["occupied_per_batch"], info["q_per_batch"], owned=owned)
        assert sum(ta * tj for _, ta, tj in sched) == info["pairs_transformed"]
