"""The multi-rank path on CPU: two gloo ranks each take their own lights and
build them with the oracle; the union equals the single-rank build, and the
timing reduction takes the max time and the summed units."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    from paper_2601_01660_b300 import scenes, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.cube_scene(200, seed=3)
    lights = scenes.four_lights()
    mine = shard.lights_for_rank(lights, rank, world)
    tau = oracle.build_tau(sc, mine, 8, 8, scenes.radii_linear(0.1, 8, 4))
    t, u = shard.reduce_step_timing(10.0 + rank, 100.0 * (rank + 1))
    out[rank] = (tau, t, u)
    dist.destroy_process_group()


def test_two_gloo_ranks_split_lights():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    import oracle
    from paper_2601_01660_b300 import scenes
    full = oracle.build_tau(scenes.cube_scene(200, seed=3), scenes.four_lights(), 8, 8,
                            scenes.radii_linear(0.1, 8, 4))
    np.testing.assert_array_equal(out[0][0], full[0::2])
    np.testing.assert_array_equal(out[1][0], full[1::2])
    for r in range(2):
        assert out[r][1] == 11.0 and out[r][2] == 300.0


def test_offset_light_is_distinct_per_rank():
    from paper_2601_01660_b300 import shard
    base = np.float32([[0, 0, 2.8]])
    a, b = shard.offset_light(base, 0), shard.offset_light(base, 3)
    assert a[0, 0] == 0.0 and b[0, 0] == np.float32(0.75) and base[0, 0] == 0.0
