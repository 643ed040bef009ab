"""The multi-process paths on CPU (gloo, world size 2): the benchmark's
barrier and max-over-ranks timing, and Merge Peaks across ranks in the
z-slab form (each rank the strict 26-neighbour maxima of its own slab's
output planes) against the oracle's Find Peaks on the whole map."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _local_maxima(s, zr, box):
    """Strict 26-neighbour maxima (ties to the lower linear index) of s with
    candidates in planes zr and neighbours inside box (a brute-force list)."""
    Z, Y, X = s.shape
    z0, z1, y0, y1, x0, x1 = box
    out_i, out_v = [], []
    for z in range(*zr):
        for y in range(y0, y1):
            for x in range(x0, x1):
                v, i = s[z, y, x], (z * Y + y) * X + x
                ok = True
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if (dz, dy, dx) == (0, 0, 0) or not (z0 <= zz < z1 and y0 <= yy < y1 and x0 <= xx < x1):
                                continue
                            o, j = s[zz, yy, xx], (zz * Y + yy) * X + xx
                            if o > v or (o == v and j < i):
                                ok = False
                if ok:
                    out_i.append(i)
                    out_v.append(v)
    return np.array(out_i, dtype=np.int64), np.array(out_v, dtype=np.float32)


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank), TTM_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    try:
        import bench
        import torch.distributed as dist
        from paper_2408_02398_gb300 import dist as tdist
        from paper_2408_02398_gb300 import synth
        w, r, _ = bench.dist_setup()
        assert (w, r) == (ws, rank)
        bench.barrier(w)
        t = bench.max_over_ranks(1.5 + rank, w, "cpu")
        # a smooth random map, its valid box, and this rank's slab of output planes
        shape = (24, 20, 22)
        s = synth.normals(77, synth.STREAM_MISC, int(np.prod(shape))).reshape(shape).astype(np.float32)
        s = (s + np.roll(s, 1, 0) + np.roll(s, 1, 1) + np.roll(s, 1, 2)).astype(np.float32)
        box = (3, 21, 2, 18, 4, 19)
        edges = np.linspace(box[0], box[1], ws + 1).astype(int)
        ci, cv = _local_maxima(s, (edges[rank], edges[rank + 1]), box)
        idx, val = tdist.gather_merge_peaks(ci, cv, shape, 25, 3.5)
        q.put((rank, t, idx.tolist(), val.tolist()))
        dist.destroy_process_group()
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None))


def test_gloo_two_ranks_timing_and_merge_peaks():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle as O
    from paper_2408_02398_gb300 import build as B
    from paper_2408_02398_gb300 import synth
    B.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ws, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q), daemon=True) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=240) for _ in range(ws)]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    for r in res:
        assert r[1] != "error", r
    shape = (24, 20, 22)
    s = synth.normals(77, synth.STREAM_MISC, int(np.prod(shape))).reshape(shape).astype(np.float32)
    s = (s + np.roll(s, 1, 0) + np.roll(s, 1, 1) + np.roll(s, 1, 2)).astype(np.float32)
    ref_i, ref_v = O.find_peaks(s.astype(np.float64), (3, 21, 2, 18, 4, 19), 25, 3.5)
    for rank, t, idx, val in res:
        assert t == 2.5                                   # max over ranks of 1.5 + rank
        assert idx == [int(i) for i in ref_i]             # the whole-map Find Peaks
        assert np.allclose(val, ref_v.astype(np.float32))
