"""Small cases for kernel profiles (ncu captures), run as

    python -m paper_2408_02398_gb300.profile_cases quaternion Z,Y,X REPS
    python -m paper_2408_02398_gb300.profile_cases correlate N

quaternion: a d' = 4 plan (n = 4, 16^3 template, r = 7, 24 x 64 field
rotations) on a Z x Y x X white-noise tomogram; one correlation, then REPS
timed calls of the quaternion maximiser (CUDA events), so that a capture of
the maximiser kernel can skip the first call and take the next.
correlate: the whole d' = 3 path of order N (default 2) on a 128 x 512 x 512
white-noise tomogram with a 40^3 template (r = 16, 24 x 16 field rotations,
FP64 local sums), run twice, for per-kernel DRAM counters of one call."""
import sys

import numpy as np


def quaternion(shape, reps: int) -> float:
    import torch
    from . import build, synth
    build.build()
    from . import ttm
    ctx = ttm.Context(0)
    tmpl = synth.gaussian_blob_template(16, seed=5)
    p = ttm.params(order_n=4, mask_radius=7.0, n_rot_base=64, dprime=4)
    m = ttm.Matcher(ctx, tmpl, p, shape)
    tomo = torch.as_tensor(synth.normals(3, 1, int(np.prod(shape))).reshape(shape).astype(np.float32), device="cuda")
    m.run(tomo)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ttm.ttm_peak_map(m.plan, m.C, m.score, m.orient, m.frob)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    print("peak map %.3f ms per call, %d voxels" % (ms, int(np.prod(shape))))
    return ms


def correlate(order_n: int) -> None:
    import torch
    from . import build, synth
    build.build()
    from . import ttm
    shape = (128, 512, 512)
    tomo = synth.normals(5, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(40, seed=5)
    ctx = ttm.Context(0)
    p = ttm.params(order_n=order_n, mask_radius=16, n_rot_base=16)
    m = ttm.Matcher(ctx, tmpl, p, shape)
    d = torch.as_tensor(tomo, device="cuda")
    for _ in range(2):
        m.run(d)
    torch.cuda.synchronize()
    print("ok", m.score.float().mean().item())


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "quaternion"
    if case == "quaternion":
        zyx = tuple(int(v) for v in (sys.argv[2] if len(sys.argv) > 2 else "64,256,256").split(","))
        reps = int(sys.argv[3]) if len(sys.argv) > 3 else 3
        quaternion(zyx, reps)
    elif case == "correlate":
        correlate(int(sys.argv[2]) if len(sys.argv) > 2 else 2)
    else:
        raise SystemExit("unknown case %r" % case)
