"""bench.py's multi-rank host logic on CPU: two gloo ranks, a barrier, and
the step time reduced as the maximum over ranks (no data-path collective);
and the row bands of one stream (--split rows): each rank's band, and all
bands together covering every row exactly once."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench

    w, r, local = bench.dist_setup()
    bench.dist_barrier(w)
    m = bench.dist_max(10.0 + 5.0 * r, w)
    bench.dist_barrier(w)
    import torch.distributed as dist

    dist.destroy_process_group()
    q.put((r, w, local, m))


def test_two_ranks_take_the_max_step_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2, 0, 15.0), (1, 2, 1, 15.0)]


def test_single_process_needs_no_process_group():
    import bench

    assert bench.dist_max(3.5, 1) == 3.5
    bench.dist_barrier(1)


def _band_rank_main(rank, world, port, H, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist

    w, r, _ = bench.dist_setup()
    mine = bench.band_of(r, w, H)
    got = [None] * w
    dist.all_gather_object(got, mine)  # host-side check only: the data path has no collective
    dist.destroy_process_group()
    q.put((r, mine, got))


def test_two_ranks_own_disjoint_bands_that_cover_the_frame():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    H = 4097  # odd: the first band takes the extra row
    procs = [ctx.Process(target=_band_rank_main, args=(r, 2, port, H, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == (0, 2049) and res[1][1] == (2049, 2048)
    for _, _, allb in res:
        assert allb == [(0, 2049), (2049, 2048)]


def test_bands_cover_every_row_once():
    import bench

    for H in (1, 2, 7, 100, 4096):
        for world in range(1, 9):
            if world > H:
                continue
            bands = [bench.band_of(r, world, H) for r in range(world)]
            covered = [row for r0, n in bands for row in range(r0, r0 + n)]
            assert covered == list(range(H)), (H, world)
            assert max(n for _, n in bands) - min(n for _, n in bands) <= 1
