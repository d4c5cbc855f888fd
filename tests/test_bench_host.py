"""Host-side logic of bench.py: the algorithmic-byte model, the replica
sharding and the max-over-ranks timing reduction (world size 2, gloo, CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_algorithmic_bytes_model():
    info = {"n_vertices": 1000, "mean_degree": 6.0}
    # M = 10, B = 16: per vertex-field 10 * (56/16 + 32) + 12/16 bytes
    b = bench.algorithmic_bytes_per_step([info], [16], [10])
    assert b == pytest.approx(1000 * 16 * (10 * (56 / 16 + 32) + 12 / 16))
    # B = 1 single field: the operator is not amortized
    assert bench.algorithmic_bytes_per_step([info], [1], [10]) == pytest.approx(1000 * (10 * (56 + 32) + 12))


def test_replica_seeds_are_distinct():
    assert len({bench.shard_seed(r) for r in range(8)}) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 3.0], world)
    out[rank] = vals
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == [2.0, 5.0, 3.0]
    assert out[1] == [2.0, 5.0, 3.0]
    assert bench.max_over_ranks([7.0], 1) == [7.0]


def test_cpu_baseline_on_all_cores_counts_every_march():
    """The all-cores oracle baseline runs every (mesh, field) march once, in
    spawned processes (one thread each), and reports the cores it used."""
    from paper_2608_03587_b300 import workloads as W
    wl = W.batched_fibers(n_meshes=2, fields_per_mesh=2, n_min=800, ratio=1.5, seed=4)
    r = bench.cpu_baseline_all_cores(wl, 2, 2, cores=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert "%d vertex-steps" % sum(m.n_vertices * 2 for m in wl.meshes) in r["sample"]


def test_traffic_ratio_covers_every_autotuned_tile_and_dataflow_shape():
    """Every tile-staged and dataflow launch shape the autotuner can keep on
    the bench batch (ring slots 3 or 2 and either walk; per-CTA chunks with
    skips 4, 8, 16 reversed or 8 forward, contiguous ranges either way) maps
    to a captured DRAM-traffic ratio, and every stored ratio to such a shape."""
    import bench
    keys = set()
    for fw in (0, 1):
        for slots in (3, 2):
            keys.add(bench.traffic_shape_key("march_tile_kernel", 1,
                                             {"forward_walk": fw, "tile_slots_used": slots}))
        for skip in ((4, 8, 16) if fw == 0 else (8,)):
            keys.add(bench.traffic_shape_key("march_flow_kernel", 3,
                                             {"forward_walk": fw, "flow_ranges": 0, "flow_skip": skip}))
        keys.add(bench.traffic_shape_key("march_flow_kernel", 3, {"forward_walk": fw, "flow_ranges": 1, "flow_skip": 8}))
    assert keys == set(bench.TRAFFIC_RATIO)
    assert all(0.9 < r < 1.05 for r in bench.TRAFFIC_RATIO.values())
    assert bench.traffic_shape_key("march_kernel<float,16>", 0, {}) not in bench.TRAFFIC_RATIO
