"""GPU parity: every step of the CUDA path, called through the C ABI, against
the FP64 oracle on the same seeded inputs, element by element, at sizes
that span several tiles and leave ragged tails.

Tolerances: C maps max abs error <= 2e-5 (FP32 FFT correlation of values
|C| <= 1), w relative 1e-5, score abs error <= 1e-4 (FP32), orientation <=
1 degree where the maximum is well separated (best minus second-best
distinct local maximum > 1e-3 |s|), peak lists bit-exact.

The local sums of Eq. 2 have two arithmetics on the GPU, FP64 and
double-float (pairs of FP32 numbers, ~48-bit significand); every test of the
correlation runs both (LOCALSUMS) against the same FP64 oracle values."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_TOL = 2e-5
S_TOL = 1e-4
W_TOL = 1e-5
ANG_TOL_DEG = 1.0
# TTM_LOCALSUM_FP64, TTM_LOCALSUM_DF64
LOCALSUMS = [0, 1]


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


def oracle_field(tmpl, r, n, n_base):
    m, _ = O.mask(tmpl.shape, r)
    tp, _ = O.normalise_template(tmpl, m)
    return O.tensor_field(tp, O.rotation_set(n_base), n, 3)


def well_defined(res):
    """Voxels whose orientation is defined to well below a degree: the best
    local maximum beats every distinct other one by > 1e-3 |s| and the
    maximum is curved (smallest curvature > 1e-3 ||C||_F)."""
    s, sec, curv, F = res["score"], res["second"], res["curv"], res["F"]
    return ((s - sec) > 1e-3 * np.abs(s)) & (curv > 1e-3 * F)


def angle_deg(u, v):
    d = np.clip(np.abs(np.sum(u * v, axis=-1)), 0, 1)
    return np.degrees(np.arccos(d))


# ------------------------------------------------------------- field --

@pytest.mark.parametrize("N,r,n", [(9, 3.0, 2), (16, 7.0, 4), (11, 4.0, 6)])
def test_tensor_field_matches_oracle(T, ctx, N, r, n):
    # the ABI takes a float32 template: give the oracle the same values
    tmpl = synth.gaussian_blob_template(N, seed=100 + N).astype(np.float32).astype(np.float64)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=32)
    K = T.ttm_num_components(n)
    d_field = torch.empty((K, N, N, N), dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, d_field)
    torch.cuda.synchronize()
    ref = oracle_field(tmpl, r, n, 32)
    got = d_field.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


# --------------------------------------------------------- correlate --

CASES = [
    # shape (Z, Y, X), template N, r, n
    ((24, 20, 28), 7, 3.0, 2),
    ((21, 20, 28), 8, 3.0, 4),
    ((32, 30, 36), 9, 4.0, 6),
    ((9, 9, 10), 9, 4.0, 2),      # volume as small as the template (one valid voxel row)
]


def run_gpu(T, ctx, tomo, field, p, localsum=0):
    plan = T.Plan(ctx, dev(field, torch.float64), p, tomo.shape)
    T.ttm_plan_set_localsum(plan, localsum)
    K = field.shape[0]
    d_C = torch.empty((K,) + tomo.shape, dtype=torch.float32, device="cuda")
    T.ttm_correlate(plan, dev(tomo), d_C)
    d_w = torch.empty(tomo.shape, dtype=torch.float32, device="cuda")
    T.ttm_plan_copy_w(plan, d_w)
    d_s = torch.empty(tomo.shape, dtype=torch.float32, device="cuda")
    d_u = torch.empty((3,) + tomo.shape, dtype=torch.float32, device="cuda")
    d_F = torch.empty(tomo.shape, dtype=torch.float32, device="cuda")
    T.ttm_peak_map(plan, d_C, d_s, d_u, d_F)
    torch.cuda.synchronize()
    return plan, d_C, d_w, d_s, d_u, d_F


@pytest.mark.parametrize("localsum", LOCALSUMS)
@pytest.mark.parametrize("shape,N,r,n", CASES)
def test_correlate_periodic_all_voxels(T, ctx, shape, N, r, n, localsum):
    """C and w on the whole grid against the oracle's periodic direct sums."""
    tomo = synth.normals(7 + N, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(N, seed=N)
    field = oracle_field(tmpl, r, n, 16)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=16)
    plan, d_C, d_w, d_s, d_u, d_F = run_gpu(T, ctx, tomo, field, p, localsum)
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    w, _, _ = O.local_w(pr.g, pr.m, None, periodic=True, floor=pr.floor)
    Cref = O.correlate(pr.g, field, None, periodic=True, w=w)
    got_w = d_w.cpu().numpy().ravel()
    assert np.abs(got_w - w).max() <= W_TOL * np.abs(w).max()
    got = d_C.cpu().numpy().reshape(field.shape[0], -1)
    assert np.abs(got - Cref).max() <= C_TOL * max(1.0, np.abs(Cref).max())
    # Frobenius proxy
    F = O.frobenius(Cref, n)
    assert np.abs(d_F.cpu().numpy().ravel() - F).max() <= C_TOL * max(1.0, F.max()) * 3


REG_CASES = [
    # lengths with register-resident FFT kernels (64, 128, 200, 256, 512) on every axis
    ((200, 64, 128), 9, 4.0, 4),
    ((64, 256, 64), 8, 3.0, 2),
    ((128, 128, 256), 11, 5.0, 6),
    ((12, 512, 512), 9, 4.0, 2),
    # double-float three-level kernels: 8*5*5 on the x and y passes, 8*8*8 and 8*8*4 on the
    # fused z pass (8*8*4 and 8*4*4 on x and y are in the cases above)
    ((16, 200, 200), 9, 4.0, 2),
    ((512, 16, 24), 9, 4.0, 2),
    ((256, 16, 24), 9, 4.0, 2),
]


@pytest.mark.parametrize("localsum", LOCALSUMS)
@pytest.mark.parametrize("shape,N,r,n", REG_CASES)
def test_correlate_register_lengths(T, ctx, shape, N, r, n, localsum):
    """C, w, score at sampled voxels (periodic) for the register FFT lengths."""
    V = int(np.prod(shape))
    tomo = synth.normals(11 + N, 1, V).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(N, seed=N + 1)
    field = oracle_field(tmpl, r, n, 16)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=16)
    plan, d_C, d_w, d_s, d_u, d_F = run_gpu(T, ctx, tomo, field, p, localsum)
    rng = np.random.default_rng(N)
    vox = np.sort(rng.choice(V, size=1500, replace=False))
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=True, floor=pr.floor)
    Cref = O.correlate(pr.g, field, vox, periodic=True, w=w)
    assert np.abs(d_w.cpu().numpy().ravel()[vox] - w).max() <= W_TOL * np.abs(w).max()
    K = field.shape[0]
    got = d_C.cpu().numpy().reshape(K, -1)[:, vox]
    assert np.abs(got - Cref).max() <= C_TOL * max(1.0, np.abs(Cref).max())
    s, _, _ = O.maximise(Cref, n, 3, nsamples=20000)
    assert np.abs(d_s.cpu().numpy().ravel()[vox] - s).max() <= S_TOL


@pytest.mark.parametrize("localsum", LOCALSUMS)
def test_local_sums_with_cancellation(T, ctx, localsum):
    """Local sums on 512-point x and y axes for a tomogram 50 + unit noise.
    The filter keeps the offset and leaves a noise variance of about 0.085,
    so S2 - S1^2/M cancels about four and a half digits of S2: FP32 local
    sums would miss w by ~1e-3, the FP64 and double-float ones must still
    match the oracle's w to the FP32 tolerance at sampled voxels."""
    shape = (12, 512, 512)
    V = int(np.prod(shape))
    tomo = (50.0 + synth.normals(21, 1, V)).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(9, seed=4)
    field = oracle_field(tmpl, 4.0, 2, 4)
    p = T.params(order_n=2, mask_radius=4.0, n_rot_base=4)
    plan, d_C, d_w, d_s, d_u, d_F = run_gpu(T, ctx, tomo, field, p, localsum)
    vox = np.sort(np.random.default_rng(5).choice(V, size=1500, replace=False))
    pr = O.Prepared(tomo.astype(np.float64), tmpl, 4.0)
    w, S1, S2 = O.local_w(pr.g, pr.m, vox, periodic=True, floor=pr.floor)
    # the cancellation the case is built for
    assert np.min((S2 - S1 ** 2 / pr.M) / S2) < 1e-4
    assert np.abs(d_w.cpu().numpy().ravel()[vox] - w).max() <= W_TOL * np.abs(w).max()


@pytest.mark.parametrize("n", [2, 4, 6])
def test_peak_map_random_tensors(T, ctx, n):
    """Maximiser on normalised random tensors: score within 1e-4 of the
    oracle's dense-sampling + Newton maximum at every voxel."""
    K = T.ttm_num_components(n)
    shape = (4, 50, 50)
    V = int(np.prod(shape))
    C = synth.random_tensors(1000 + n, V, K).T.copy()      # [K][V]
    C /= O.frobenius(C, n)[None, :]                        # ||C||_F = 1
    tmpl = synth.gaussian_blob_template(3, seed=1)
    field = oracle_field(tmpl, 1.0, n, 4)
    p = T.params(order_n=n, mask_radius=1.0, n_rot_base=4)
    plan = T.Plan(ctx, dev(field, torch.float64), p, shape)
    d_s = torch.empty(shape, dtype=torch.float32, device="cuda")
    d_u = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
    d_F = torch.empty(shape, dtype=torch.float32, device="cuda")
    T.ttm_peak_map(plan, dev(C.reshape((K,) + shape)), d_s, d_u, d_F)
    torch.cuda.synchronize()
    sv = np.arange(V)[:: max(1, V // 3000)]
    s, u, sec, curv = O.maximise(C[:, sv], n, 3, nsamples=20000, with_curvature=True)
    gs = d_s.cpu().numpy().ravel()[sv]
    gu = d_u.cpu().numpy().reshape(3, -1)[:, sv].T
    err = np.abs(gs - s)
    assert err.max() <= S_TOL, (err.max(), int((err > S_TOL).sum()))
    sep = well_defined({"score": s, "second": sec, "curv": curv, "F": np.ones_like(s)})
    assert angle_deg(gu[sep], u[sep]).max() <= ANG_TOL_DEG
    assert np.all(gu[:, 2] >= 0)
    assert np.abs(d_F.cpu().numpy().ravel() - 1.0).max() < 1e-5


@pytest.mark.parametrize("localsum", LOCALSUMS)
def test_degenerate_inputs(T, ctx, localsum):
    """Constant tomogram: where the mask ball stays clear of the zero-padded
    outer layer the local variance is zero -> w = 0 -> C = 0, score 0;
    next to the outer layer w follows the oracle."""
    shape = (16, 16, 20)
    tmpl = synth.gaussian_blob_template(7, seed=3)
    field = oracle_field(tmpl, 3.0, 2, 4)
    p = T.params(order_n=2, mask_radius=3.0, n_rot_base=4)
    tomo = np.full(shape, 2.5, np.float32)
    plan, d_C, d_w, d_s, d_u, d_F = run_gpu(T, ctx, tomo, field, p, localsum)
    z0, z1, y0, y1, x0, x1 = plan.valid_box()
    inner = (slice(z0 + 1, z1 - 1), slice(y0 + 1, y1 - 1), slice(x0 + 1, x1 - 1))
    assert np.all(d_w.cpu().numpy()[inner] == 0)
    assert np.all(d_s.cpu().numpy()[inner] == 0)
    assert np.all(d_C.cpu().numpy()[(slice(None),) + inner] == 0)
    pr = O.Prepared(tomo.astype(np.float64), tmpl, 3.0)
    v = O.valid_voxels(shape, tmpl.shape)
    w, _, _ = O.local_w(pr.g, pr.m, v, False, pr.floor)
    got = d_w.cpu().numpy().ravel()[v]
    assert np.abs(got - w).max() <= 1e-5 * np.abs(w).max()


def test_errors_are_reported(T, ctx):
    tmpl = synth.gaussian_blob_template(7, seed=3)
    field = dev(oracle_field(tmpl, 3.0, 2, 4), torch.float64)
    p = T.params(order_n=2, mask_radius=3.0, n_rot_base=4)
    with pytest.raises(T.TTMError) as e:
        T.Plan(ctx, field, p, (17, 16, 16))          # 17 is not 7-smooth
    assert e.value.code == 2
    with pytest.raises(T.TTMError) as e:
        T.Plan(ctx, field, p, (6, 16, 16))           # smaller than the template
    assert e.value.code == 2
    with pytest.raises(ValueError):   # a d' = 3 field (6 components) for a d' = 4 plan (10)
        T.Plan(ctx, field, T.params(order_n=2, mask_radius=3.0, dprime=4), (16, 16, 16))
    with pytest.raises(T.TTMError) as e:
        T.Plan(ctx, field, T.params(order_n=2, mask_radius=3.5), (16, 16, 16))  # mask does not fit 7^3
    assert e.value.code == 1
    L = T.lib()
    assert L.ttm_correlate(None, None, None, None) == 1


# -------------------------------------------------------------- TM --

def test_tm_matches_oracle(T, ctx):
    shape = (20, 21, 24)
    N, r = 7, 3.0
    tomo = synth.normals(55, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(N, seed=55)
    quats = np.vstack([O.cube_rotations()[:6], synth.shoemake_quats(synth.uniforms(55, 9, 6))])
    p = T.params(order_n=2, mask_radius=r)
    d_best = torch.empty(shape, dtype=torch.float32, device="cuda")
    d_idx = torch.empty(shape, dtype=torch.int32, device="cuda")
    T.tm_correlate(ctx, dev(tomo), dev(tmpl), p, quats, d_best, d_idx)
    torch.cuda.synchronize()
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    w, _, _ = O.local_w(pr.g, pr.m, None, periodic=True, floor=pr.floor)
    best, idx = O.tm(pr.g, pr.tp, quats, None, periodic=True, w=w)
    gb = d_best.cpu().numpy().ravel()
    gi = d_idx.cpu().numpy().ravel()
    assert np.abs(gb - best).max() <= C_TOL
    # the arg-max index is unique wherever the best two rotations differ clearly
    allc = np.stack([O.correlate(pr.g, O.rotate_template(pr.tp, q)[None], None, True, w)[0] for q in quats])
    srt = np.sort(allc, axis=0)
    clear = (srt[-1] - srt[-2]) > 1e-4
    assert np.array_equal(gi[clear], idx[clear])


def test_tm_finds_planted_copy_with_lncc_one(T, ctx):
    """A copy of the template rotated by a quarter-turn, alone in a zero
    volume, gives LNCC 1 at its centre for that rotation (Eqs. 1-5)."""
    N, r = 9, 4.0
    tmpl = synth.gaussian_blob_template(N, seed=77)
    s = math.sqrt(0.5)
    quats = np.array([[1, 0, 0, 0], [s, 0, 0, s], [s, 0, 0, -s], [0, 1, 0, 0.0]])
    vol = np.zeros((24, 24, 28), np.float32)
    rot = O.rotate_template(tmpl, quats[1]).astype(np.float32)
    c0 = (12, 11, 13)
    h = N // 2
    vol[c0[0] - h:c0[0] + h + 1, c0[1] - h:c0[1] + h + 1, c0[2] - h:c0[2] + h + 1] = rot
    p = T.params(order_n=2, mask_radius=r)
    d_best = torch.empty(vol.shape, dtype=torch.float32, device="cuda")
    d_idx = torch.empty(vol.shape, dtype=torch.int32, device="cuda")
    T.tm_correlate(ctx, dev(vol), dev(tmpl), p, quats, d_best, d_idx)
    torch.cuda.synchronize()
    assert d_idx[c0].item() == 1
    assert abs(d_best[c0].item() - 1.0) < 1e-4


# ----------------------------------------------------- find peaks --

def test_find_peaks_host_logic_bit_exact(T, ctx):
    shape = (20, 24, 28)
    rng = np.random.default_rng(5)
    s = rng.random(shape).astype(np.float32)
    s[5:8, 5:8, 5:8] = 2.0     # a plateau: one peak at its lowest index
    tmpl = synth.gaussian_blob_template(5, seed=1)
    field = oracle_field(tmpl, 2.0, 2, 4)
    plan = T.Plan(ctx, dev(field, torch.float64), T.params(order_n=2, mask_radius=2.0, n_rot_base=4), shape)
    box = plan.valid_box()
    for P, md in [(10, 4.0), (50, 2.5), (0, 1.0), (1000, 1.0)]:
        gi, gv = T.ttm_find_peaks(plan, dev(s), P, md)
        oi, ov = O.find_peaks(s.astype(np.float64), box, P, md)
        assert np.array_equal(gi, oi)
        assert np.array_equal(gv.astype(np.float64), ov)


# ------------------------------------------------------- end to end --

@pytest.fixture(scope="module")
def small(T, ctx):
    """64^3 white noise, 16^3 six-Gaussian template, r = 7, n = 2, four copies
    at amplitude 0.5; GPU path with its own field, oracle with its own."""
    wl = synth.workload_small()
    p = T.params(order_n=2, mask_radius=wl.mask_radius, n_rot_base=2048)
    m = T.Matcher(ctx, wl.template, p, wl.tomo.shape)
    m.run(dev(wl.tomo))
    torch.cuda.synchronize()
    res = O.ttm(wl.tomo, wl.template, wl.mask_radius, 2, O.rotation_set(2048))
    return wl, m, res


def test_small_workload_field(T, small):
    wl, m, res = small
    got = m.field.cpu().numpy()
    assert np.abs(got - res["T"]).max() <= 1e-12 * np.abs(res["T"]).max()


def test_small_workload_maps(T, small):
    wl, m, res = small
    v = res["vox"]
    K = res["C"].shape[0]
    gC = m.C.cpu().numpy().reshape(K, -1)[:, v]
    assert np.abs(gC - res["C"]).max() <= C_TOL
    gs = m.score.cpu().numpy().ravel()[v]
    assert np.abs(gs - res["score"]).max() <= S_TOL
    gF = m.frob.cpu().numpy().ravel()[v]
    assert np.abs(gF - res["F"]).max() <= C_TOL * 3
    gu = m.orient.cpu().numpy().reshape(3, -1)[:, v].T
    sep = well_defined(res)
    assert sep.mean() > 0.9
    assert angle_deg(gu[sep], res["orient"][sep]).max() <= ANG_TOL_DEG
    # at the planted centres
    Z, Y, X = wl.tomo.shape
    pos = {int(x): i for i, x in enumerate(v)}
    for c in wl.planted.centres:
        i = pos[int((c[0] * Y + c[1]) * X + c[2])]
        assert abs(gs[i] - res["score"][i]) <= S_TOL
        if sep[i]:
            assert angle_deg(gu[i], res["orient"][i]) <= ANG_TOL_DEG


def peak_groups(ov, tol):
    """Runs of consecutive peaks whose values lie within tol of the next one:
    inside a run the order may legitimately differ between two maps that
    agree to tol/2."""
    out, j = [], 0
    while j < len(ov):
        k = j
        while k + 1 < len(ov) and ov[k] - ov[k + 1] <= tol:
            k += 1
        out.append((j, k + 1))
        j = k + 1
    return out


def test_small_workload_peaks(T, small):
    """Peak lists of the GPU score and Frobenius maps against the oracle's
    (16 peaks asked, the first 12 compared). Every peak whose value is more
    than 2 * S_TOL from its neighbours sits at the same rank with the same
    index; a run of peaks closer than that must hold the same set of
    indices. Every oracle peak within 4 voxels of a planted centre is
    among the compared ones and is matched that way."""
    wl, m, res = small
    Z, Y, X = wl.tomo.shape
    box = m.plan.valid_box()
    cen = np.asarray(wl.planted.centres, dtype=float)
    for key, gmap in (("score", m.score), ("F", m.frob)):
        full = np.full(Z * Y * X, -np.inf)
        full[res["vox"]] = res[key]
        oi, ov = O.find_peaks(full.reshape(Z, Y, X), box, 16, 2 * wl.mask_radius)
        gi, gv = T.ttm_find_peaks(m.plan, gmap, 16, 2 * wl.mask_radius)
        assert len(gi) == len(oi) == 16
        compared = 0
        for j, k in peak_groups(ov, 2 * S_TOL):
            if j >= 12 or k == len(ov):
                break   # a run cut by the list end may continue past it
            assert set(gi[j:k]) == set(oi[j:k]), (key, j, gi[j:k], oi[j:k])
            compared = k
        assert compared >= 10, (key, compared)
        pos = {int(i): v for i, v in zip(gi, gv)}
        for i, v in zip(oi[:compared], ov[:compared]):
            assert abs(pos[int(i)] - v) <= S_TOL
        zyx = np.stack([oi // (Y * X), (oi // X) % Y, oi % X], axis=1).astype(float)
        near = np.min(np.linalg.norm(zyx[:, None, :] - cen[None, :, :], axis=2), axis=1) <= 4.0
        assert near[:compared].sum() >= 2 and near[compared:12].sum() == 0, (key, near)


# ---------------------------------------------- full size, bench config --

@pytest.fixture(scope="module")
def fullsize(T, ctx):
    """512 x 512 x 200 low-passed noise, 40^3 template, r = 16, n = 4, 300
    planted copies: the shapes and launch configuration the benchmark
    times. The oracle is evaluated voxel by voxel at 10 000 random valid
    voxels plus every planted centre. The quadrature is reduced to 24 x 64
    rotations on both sides (the per-tomogram kernels do not depend on it)."""
    wl = synth.workload_order4()
    n, r = wl.order_n, wl.mask_radius
    p = T.params(order_n=n, mask_radius=r, n_rot_base=64)
    m = T.Matcher(ctx, wl.template, p, wl.tomo.shape)
    Z, Y, X = wl.tomo.shape
    valid = O.valid_voxels(wl.tomo.shape, wl.template.shape)
    rng = np.random.default_rng(3)
    cent = np.array([(c[0] * Y + c[1]) * X + c[2] for c in wl.planted.centres], dtype=np.int64)
    vox = np.unique(np.concatenate([valid[rng.choice(valid.size, 10000, replace=False)], cent]))
    res = O.ttm(wl.tomo, wl.template, r, n, O.rotation_set(64), vox)
    return wl, m, vox, cent, res


@pytest.mark.parametrize("localsum", LOCALSUMS)
def test_fullsize_order4_sampled(T, fullsize, localsum):
    """The benchmark's workload in both local-sum arithmetics: field, w, C,
    score and (where well defined) orientation at >= 10 000 sampled voxels
    and at all 300 planted centres."""
    wl, m, vox, cent, res = fullsize
    T.ttm_plan_set_localsum(m.plan, localsum)
    m.run(dev(wl.tomo))
    d_w = torch.empty(wl.tomo.shape, dtype=torch.float32, device="cuda")
    T.ttm_plan_copy_w(m.plan, d_w)
    torch.cuda.synchronize()
    assert vox.size >= 10000 and np.isin(cent, vox).all()
    assert np.abs(m.field.cpu().numpy() - res["T"]).max() <= 1e-12 * np.abs(res["T"]).max()
    gw = d_w.cpu().numpy().ravel()[vox]
    assert np.abs(gw - res["w"]).max() <= W_TOL * np.abs(res["w"]).max()
    K = res["C"].shape[0]
    gC = m.C.cpu().numpy().reshape(K, -1)[:, vox]
    assert np.abs(gC - res["C"]).max() <= C_TOL
    gs = m.score.cpu().numpy().ravel()[vox]
    err = np.abs(gs - res["score"])
    assert err.max() <= S_TOL, (err.max(), int((err > S_TOL).sum()))
    gF = m.frob.cpu().numpy().ravel()[vox]
    assert np.abs(gF - res["F"]).max() <= 3 * C_TOL
    gu = m.orient.cpu().numpy().reshape(3, -1)[:, vox].T
    ok = well_defined(res)
    assert ok.mean() > 0.5
    assert angle_deg(gu[ok], res["orient"][ok]).max() <= ANG_TOL_DEG
