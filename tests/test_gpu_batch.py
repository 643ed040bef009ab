"""Zero-padded working grids, the FFT autotuner, and batched TTM (many
tomograms of uneven sizes times several templates in one captured graph):
padded plans against unpadded ones and against the oracle, the batch
against per-pair plans (identical kernels: bit-exact) and the oracle."""
import json

import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

C_TOL = 2e-5
S_TOL = 1e-4


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_02398_gb300 import build
    build.build()
    from paper_2408_02398_gb300 import ttm
    return ttm


@pytest.fixture(scope="module")
def ctx(T):
    return T.Context(0)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def smooth7(L):
    for r in (2, 3, 5, 7):
        while L % r == 0:
            L //= r
    return L == 1


def gpu_field(T, ctx, tmpl, p):
    K = T.ttm_num_components(p.order_n)
    f = torch.empty((K,) + tmpl.shape, dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, f)
    return f


def run_plan(T, ctx, field, p, tomo, work_shape=None, localsum=0):
    plan = T.Plan(ctx, field, p, tomo.shape, work_shape=work_shape)
    T.ttm_plan_set_localsum(plan, localsum)
    K = field.shape[0]
    Zw, Yw, Xw = plan.shape
    d_C = torch.empty((K, Zw, Yw, Xw), device="cuda")
    T.ttm_correlate(plan, dev(tomo), d_C)
    d_s = torch.empty((Zw, Yw, Xw), device="cuda")
    d_u = torch.empty((3, Zw, Yw, Xw), device="cuda")
    d_F = torch.empty((Zw, Yw, Xw), device="cuda")
    T.ttm_peak_map(plan, d_C, d_s, d_u, d_F)
    torch.cuda.synchronize()
    return plan, d_C, d_s, d_u, d_F


def box_slice(b):
    return (slice(b[0], b[1]), slice(b[2], b[3]), slice(b[4], b[5]))


def test_padded_plan_matches_unpadded(T, ctx):
    shape = (40, 48, 36)
    tmpl = synth.gaussian_blob_template(12, seed=3).astype(np.float32)
    p = T.params(order_n=4, mask_radius=5.0, n_rot_base=16)
    field = gpu_field(T, ctx, tmpl, p)
    tomo = synth.normals(5, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    pa, Ca, sa, ua, Fa = run_plan(T, ctx, field, p, tomo)
    pb, Cb, sb, ub, Fb = run_plan(T, ctx, field, p, tomo, work_shape=(49, 56, 45))
    b = pa.valid_box()
    assert pb.valid_box() == b
    bs = box_slice(b)
    ca = Ca[(slice(None),) + bs]
    cb = Cb[(slice(None),) + bs]
    assert (ca - cb).abs().max().item() <= C_TOL * max(1.0, ca.abs().max().item())
    assert (sa[bs] - sb[bs]).abs().max().item() <= S_TOL


def test_padded_plan_vs_oracle_prime_extents(T, ctx):
    """A 37 x 41 x 43 tomogram (prime extents, no direct FFT) on an
    autotuned working grid: C and score at valid voxels against the
    oracle's direct sums on the unpadded tomogram."""
    shape = (37, 41, 43)
    tmpl = synth.gaussian_blob_template(11, seed=4)
    r, n = 5.0, 4
    p = T.params(order_n=n, mask_radius=r, n_rot_base=16)
    m, _ = O.mask(tmpl.shape, r)
    tp, _ = O.normalise_template(tmpl, m)
    field = O.tensor_field(tp, O.rotation_set(16), n, 3)
    work = T.ttm_autotune_shape(ctx, shape)
    assert all(w >= s and smooth7(w) for w, s in zip(work, shape))
    tomo = synth.normals(6, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    plan, d_C, d_s, d_u, d_F = run_plan(T, ctx, dev(field, torch.float64), p, tomo, work_shape=work)
    b = plan.valid_box()
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    vox = O.valid_voxels(shape, tmpl.shape)
    vox = np.sort(np.random.default_rng(1).choice(vox, 600, replace=False))
    w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=False, floor=pr.floor)
    Cref = O.correlate(pr.g, field, vox, periodic=False, w=w)
    z, y, x = np.unravel_index(vox, shape)
    K = field.shape[0]
    got = d_C.cpu().numpy()[:, z, y, x]
    assert np.abs(got - Cref).max() <= C_TOL * max(1.0, np.abs(Cref).max())
    sref, _, _ = O.maximise(Cref, n, 3, nsamples=20000)
    assert np.abs(d_s.cpu().numpy()[z, y, x] - sref).max() <= S_TOL
    assert b[1] - b[0] == shape[0] - tmpl.shape[0] + 1


def test_autotune_cache_roundtrip(T, ctx, tmp_path):
    T.ttm_autotune_shape(ctx, (97, 131, 211))
    n = T.ttm_autotune_entries(ctx)
    assert n >= 3
    f = str(tmp_path / "tune.json")
    T.ttm_autotune_save(ctx, f)
    recs = json.load(open(f))
    assert len(recs) == n
    for r in recs:
        assert int(np.prod(r["rad"])) == r["L"] and r["kind"] in (0, 2)
        assert r["us_line"] > 0 or r["kind"] == 2   # double-float lengths without a register kernel are not timed
    ctx2 = T.Context(0)
    T.ttm_autotune_load(ctx2, f)
    assert T.ttm_autotune_entries(ctx2) == n
    bad = tmp_path / "bad.json"
    bad.write_text('[\n  {"L": 96, "kind": 0, "reg": 0, "W": 8, "rad": [8, 4, 2], "us_line": 0.1}\n]\n')
    with pytest.raises(T.TTMError):
        T.ttm_autotune_load(ctx2, str(bad))


SHAPES = [(37, 52, 45), (61, 40, 44), (50, 50, 50)]


@pytest.fixture(scope="module")
def batch_setup(T, ctx):
    p = T.params(order_n=4, mask_radius=5.0, n_rot_base=16)
    tmpls = [synth.gaussian_blob_template(12, seed=20 + j).astype(np.float32) for j in range(2)]
    fields = [gpu_field(T, ctx, t, p) for t in tmpls]
    tomos = [dev(synth.normals(30 + i, 1, int(np.prod(s))).reshape(s).astype(np.float32))
             for i, s in enumerate(SHAPES)]
    items, outs = [], []
    for i, s in enumerate(SHAPES):
        for j in range(2):
            sc = torch.full(s, -7.0, device="cuda")
            ori = torch.zeros((3,) + s, device="cuda")
            fr = torch.zeros(s, device="cuda")
            items.append((i, j, sc, ori, fr))
            outs.append((i, j, sc, ori, fr))
    B = T.Batch(ctx, p, fields, tomos, items, n_branches=3)
    B.run()
    torch.cuda.synchronize()
    return p, tmpls, fields, tomos, B, outs


def test_batch_matches_per_pair_plans(T, ctx, batch_setup):
    p, tmpls, fields, tomos, B, outs = batch_setup
    for i, j, sc, ori, fr in outs:
        work = B.work_shape(i)
        plan, d_C, d_s, d_u, d_F = run_plan(T, ctx, fields[j], p, tomos[i].cpu().numpy(), work_shape=work)
        b = plan.valid_box()
        bs = box_slice(b)
        assert torch.equal(sc[bs], d_s[bs])
        assert torch.equal(ori[(slice(None),) + bs], d_u[(slice(None),) + bs])
        assert torch.equal(fr[bs], d_F[bs])
        outside = torch.ones_like(sc, dtype=torch.bool)
        outside[bs] = False
        assert bool((sc[outside] == -7.0).all())


def test_batch_replay_follows_input(T, ctx, batch_setup):
    """The graph reads the tomograms at every launch: new contents, new maps."""
    p, tmpls, fields, tomos, B, outs = batch_setup
    before = outs[0][2].clone()
    tomos[0].mul_(-1.0)
    B.run()
    torch.cuda.synchronize()
    i, j, sc, ori, fr = outs[0]
    plan, d_C, d_s, d_u, d_F = run_plan(T, ctx, fields[j], p, tomos[i].cpu().numpy(), work_shape=B.work_shape(i))
    bs = box_slice(plan.valid_box())
    assert torch.equal(sc[bs], d_s[bs])
    assert not torch.equal(sc[bs], before[bs])
    tomos[0].mul_(-1.0)
    B.run()
    torch.cuda.synchronize()
    assert torch.equal(outs[0][2][bs], before[bs])


def test_batch_vs_oracle(T, ctx, batch_setup):
    """The oracle builds its own field from the same (float32) template and
    works on the host copy of the same seeded tomogram."""
    p, tmpls, fields, tomos, B, outs = batch_setup
    r, n = 5.0, 4
    ofield = {}
    for i, j, sc, ori, fr in outs[:4]:
        shape = SHAPES[i]
        tomo = synth.normals(30 + i, 1, int(np.prod(shape))).reshape(shape).astype(np.float32).astype(np.float64)
        pr = O.Prepared(tomo, tmpls[j].astype(np.float64), r)
        if j not in ofield:
            ofield[j] = O.tensor_field(pr.tp, O.rotation_set(16), n, 3)
        vox = O.valid_voxels(shape, tmpls[j].shape)
        vox = np.sort(np.random.default_rng(i + 10 * j).choice(vox, 300, replace=False))
        w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=False, floor=pr.floor)
        Cref = O.correlate(pr.g, ofield[j], vox, periodic=False, w=w)
        sref, _, _ = O.maximise(Cref, n, 3, nsamples=20000)
        z, y, x = np.unravel_index(vox, shape)
        assert np.abs(sc.cpu().numpy()[z, y, x] - sref).max() <= S_TOL


def test_batch_double_float_localsums(T, ctx, batch_setup):
    """TTM_BATCH_LOCALSUM_DF64: the batch with double-float local sums equals
    per-pair plans set to TTM_LOCALSUM_DF64 bit for bit, and its scores
    match the FP64 oracle at sampled valid voxels within the FP32 score
    tolerance."""
    p, tmpls, fields, tomos, _, _ = batch_setup
    r, n = 5.0, 4
    items = []
    for i, s in enumerate(SHAPES):
        for j in range(2):
            items.append((i, j, torch.full(s, -7.0, device="cuda"), torch.zeros((3,) + s, device="cuda"),
                          torch.zeros(s, device="cuda")))
    B = T.Batch(ctx, p, fields, tomos, items, n_branches=2, flags=T.TTM_BATCH_LOCALSUM_DF64)
    B.run()
    torch.cuda.synchronize()
    ofield = {}
    for i, j, sc, ori, fr in items:
        plan, d_C, d_s, d_u, d_F = run_plan(T, ctx, fields[j], p, tomos[i].cpu().numpy(),
                                            work_shape=B.work_shape(i), localsum=1)
        bs = box_slice(plan.valid_box())
        assert torch.equal(sc[bs], d_s[bs])
        assert torch.equal(ori[(slice(None),) + bs], d_u[(slice(None),) + bs])
        shape = SHAPES[i]
        tomo = tomos[i].cpu().numpy().astype(np.float64)
        pr = O.Prepared(tomo, tmpls[j].astype(np.float64), r)
        if j not in ofield:
            ofield[j] = O.tensor_field(pr.tp, O.rotation_set(16), n, 3)
        vox = O.valid_voxels(shape, tmpls[j].shape)
        vox = np.sort(np.random.default_rng(7 + i + 10 * j).choice(vox, 300, replace=False))
        w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=False, floor=pr.floor)
        Cref = O.correlate(pr.g, ofield[j], vox, periodic=False, w=w)
        sref, _, _ = O.maximise(Cref, n, 3, nsamples=20000)
        z, y, x = np.unravel_index(vox, shape)
        assert np.abs(sc.cpu().numpy()[z, y, x] - sref).max() <= S_TOL
        assert np.abs(d_C.cpu().numpy()[:, z, y, x] - Cref).max() <= C_TOL * max(1.0, np.abs(Cref).max())
