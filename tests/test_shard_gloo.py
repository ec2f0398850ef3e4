"""The multi-rank path on CPU: two gloo ranks each take their own lights and
build them with the oracle; the union equals the single-rank build, and the
timing reduction takes the max time and the summed units.  The row-band
split of one light set's atlas: two and three gloo ranks each build their
band with the oracle, the all-gather and reassembly of shard.banded_atlas
give every rank the full oracle atlas, and the band partition covers every
row once in whole tiles."""
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


def _band_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2601_01660_b300 import scenes, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.cube_scene(150, seed=5)
    lights = np.float32([[0, 0, 0], [0.5, -0.3, 1.0]])
    radii = scenes.radii_linear(0.1, 8, 4)
    H, W, tile, K, L = 36, 20, 8, 4, 2          # 5 tile rows, the last one partial

    def build_band(r0, r1):
        full = np.ones((L, K, H, W))
        lij = np.array([(l, i, j) for l in range(L) for i in range(r0, r1) for j in range(W)])
        T = np.exp(-oracle.build_tau_texels(sc, lights, H, W, radii, lij))
        full[lij[:, 0], :, lij[:, 1], lij[:, 2]] = T
        return torch.from_numpy(full)

    def extract(full, r0, n, slab):
        slab[:, :, :n] = full[:, :, r0:r0 + n]

    def insert(slab, q0, n, atlas):
        atlas[:, :, q0:q0 + n] = slab[:, :, :n]

    atlas = shard.banded_atlas(build_band, extract, insert,
                               lambda rows: torch.full((L, K, rows, W), float("nan"), dtype=torch.float64),
                               H, tile)
    out[rank] = atlas.numpy()
    dist.destroy_process_group()


def test_gloo_ranks_split_one_atlas_by_rows():
    import oracle
    from paper_2601_01660_b300 import scenes
    ref = oracle.build_atlas(scenes.cube_scene(150, seed=5), np.float32([[0, 0, 0], [0.5, -0.3, 1.0]]), 36, 20,
                             scenes.radii_linear(0.1, 8, 4))
    assert ref.min() < 0.9
    ctx = mp.get_context("spawn")
    for world in (2, 3):
        mgr = ctx.Manager()
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_band_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        for r in range(world):
            np.testing.assert_array_equal(out[r], ref)


def test_band_rows_partition():
    from paper_2601_01660_b300 import shard
    for H, tile, world in [(512, 8, 8), (36, 8, 2), (36, 8, 3), (40, 16, 5), (8, 8, 4), (100, 4, 7)]:
        rows = []
        for r in range(world):
            r0, r1, hb = shard.band_rows(H, tile, r, world)
            assert 0 <= r1 - r0 <= hb and hb % tile == 0 and (r1 == r0 or r0 % tile == 0)
            rows += list(range(r0, r1))
        assert rows == list(range(H))


def test_offset_light_is_distinct_per_rank():
    from paper_2601_01660_b300 import shard
    base = np.float32([[0, 0, 2.8]])
    a, b = shard.offset_light(base, 0), shard.offset_light(base, 3)
    assert a[0, 0] == 0.0 and b[0, 0] == np.float32(0.75) and base[0, 0] == 0.0
