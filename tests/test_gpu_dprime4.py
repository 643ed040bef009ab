"""GPU parity of the quaternion form (d' = 4, Sec. 3): the tensor field with
u_q = q, the correlation of its K = 10 / 35 / 84 components, and the
maximiser over unit quaternions, each against the FP64 oracle on the same
seeded inputs through the C ABI.

Tolerances: field relative 1e-12 (FP64 on both sides), C max abs error
<= 2e-5 (FP32 FFT correlation, |C| <= 1), score abs error <= 1e-4 at every
voxel of correlation maps. On i.i.d. Gaussian tensors (far more local
maxima than any correlation map) the multi-start maximiser may settle on a
lower maximum whose value is within a few 1e-4 ||C||_F of the best: at
most 1 voxel in 1000 may miss by more than 1e-4 and none by more than
1e-2 ||C||_F. Orientations are compared as rotations (angle between
R(q) and R(q')) where the maximum is well separated."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_TOL = 2e-5
S_TOL = 1e-4
ANG_TOL_DEG = 1.0


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


def oracle_field4(tmpl, r, n, n_base):
    m, _ = O.mask(tmpl.shape, r)
    tp, _ = O.normalise_template(tmpl, m)
    return O.tensor_field(tp, O.rotation_set(n_base), n, 4)


def rot_angle_deg(q1, q2):
    """rotation angle between R(q1) and R(q2), rows of unit quaternions:
    2 acos |q1 . q2| (q and -q are the same rotation)"""
    d = np.clip(np.abs(np.sum(q1 * q2, axis=-1)), 0, 1)
    return np.degrees(2 * np.arccos(d))


def well_defined(s, sec, curv, F):
    return ((s - sec) > 1e-3 * np.abs(s)) & (curv > 1e-3 * F)


def maps(T, ctx, plan, d_C, shape):
    d_s = torch.empty(shape, dtype=torch.float32, device="cuda")
    d_q = torch.empty((4,) + shape, dtype=torch.float32, device="cuda")
    d_F = torch.empty(shape, dtype=torch.float32, device="cuda")
    T.ttm_peak_map(plan, d_C, d_s, d_q, d_F)
    torch.cuda.synchronize()
    return d_s.cpu().numpy(), d_q.cpu().numpy(), d_F.cpu().numpy()


# ------------------------------------------------------------- field --

@pytest.mark.parametrize("N,r,n", [(9, 3.0, 2), (12, 5.0, 4), (9, 3.0, 6)])
def test_quaternion_field_matches_oracle(T, ctx, N, r, n):
    """K = 10, 35 and 84 (the last in three launches of 28 components)."""
    tmpl = synth.gaussian_blob_template(N, seed=200 + N).astype(np.float32).astype(np.float64)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=32, dprime=4)
    K = T.ttm_num_components(n, 4)
    assert K == {2: 10, 4: 35, 6: 84}[n]
    d_field = torch.empty((K, N, N, N), dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, d_field)
    torch.cuda.synchronize()
    ref = oracle_field4(tmpl, r, n, 32)
    got = d_field.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


# --------------------------------------------------------- correlate --

@pytest.mark.parametrize("shape,N,r,n", [((21, 20, 28), 8, 3.0, 2), ((24, 20, 30), 9, 4.0, 4),
                                         ((20, 18, 16), 7, 3.0, 6)])
def test_quaternion_correlation_and_score_match_oracle(T, ctx, shape, N, r, n):
    tomo = synth.normals(300 + n, 1, int(np.prod(shape))).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(N, seed=300 + n)
    field = oracle_field4(tmpl, r, n, 16)
    K = field.shape[0]
    p = T.params(order_n=n, mask_radius=r, n_rot_base=16, dprime=4)
    plan = T.Plan(ctx, dev(field, torch.float64), p, shape)
    d_C = torch.empty((K,) + shape, dtype=torch.float32, device="cuda")
    T.ttm_correlate(plan, dev(tomo), d_C)
    torch.cuda.synchronize()
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    vox = O.valid_voxels(shape, tmpl.shape)
    vox = np.sort(np.random.default_rng(n).choice(vox, min(400, vox.size), replace=False))
    w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=False, floor=pr.floor)
    Cref = O.correlate(pr.g, field, vox, periodic=False, w=w)
    z, y, x = np.unravel_index(vox, shape)
    got = d_C.cpu().numpy()[:, z, y, x]
    assert np.abs(got - Cref).max() <= C_TOL * max(1.0, np.abs(Cref).max())
    s, q, F = maps(T, ctx, plan, d_C, shape)
    sref, qref, sec, curv = O.maximise(Cref, n, 4, nsamples=20000, with_curvature=True)
    Fref = O.frobenius(Cref, n, 4)
    assert np.abs(s[z, y, x] - sref).max() <= S_TOL
    # |dF| <= ||dC||_F <= sqrt(sum of multiplicities = 4^n) max |dC|
    assert np.abs(F[z, y, x] - Fref).max() <= 2.0 ** n * C_TOL * max(1.0, np.abs(Cref).max())
    gq = q[:, z, y, x].T
    assert np.allclose(np.linalg.norm(gq, axis=1), 1.0, atol=1e-5)
    assert (gq[:, 0] >= 0).all()
    wd = well_defined(sref, sec, curv, Fref)
    assert wd.sum() > 20
    assert rot_angle_deg(gq[wd], qref[wd]).max() <= ANG_TOL_DEG


# --------------------------------------------------------- maximiser --

@pytest.mark.parametrize("n", [2, 4, 6])
def test_quaternion_maximiser_random_tensors(T, ctx, n):
    """||C||_F = 1 Gaussian tensors on a 4 x 50 x 50 grid (ragged against the
    256-voxel CTAs), sampled voxels against the oracle's 20000-sample +
    Newton maximiser. n = 2 takes the top eigenpair of the 4 x 4 matrix
    directly (no probes), n = 4 and 6 the probe starts."""
    K = T.ttm_num_components(n, 4)
    shape = (4, 50, 50)
    V = int(np.prod(shape))
    C = synth.random_tensors(2000 + n, V, K).T.copy()
    C /= O.frobenius(C, n, 4)[None, :]
    tmpl = synth.gaussian_blob_template(3, seed=1)
    field = oracle_field4(tmpl, 1.0, n, 4)
    p = T.params(order_n=n, mask_radius=1.0, n_rot_base=4, dprime=4)
    plan = T.Plan(ctx, dev(field, torch.float64), p, shape)
    s, q, F = maps(T, ctx, plan, dev(C.reshape((K,) + shape)), shape)
    sv = np.arange(V)[:: max(1, V // 3000)]
    sref, qref, sec, curv = O.maximise(C[:, sv], n, 4, nsamples=20000, with_curvature=True)
    gs = s.ravel()[sv]
    gq = q.reshape(4, -1)[:, sv].T
    err = sref - gs
    assert (gs - sref).max() <= 1e-5           # never above the true maximum
    assert err.max() <= 1e-2
    assert (err > S_TOL).sum() <= sv.size // 1000, (err.max(), int((err > S_TOL).sum()))
    assert np.abs(F.ravel()[sv] - 1.0).max() <= 1e-5
    ok = (err <= S_TOL) & well_defined(sref, sec, curv, np.ones_like(sref))
    assert rot_angle_deg(gq[ok], qref[ok]).max() <= ANG_TOL_DEG
    if n == 2:
        # a quadratic form has one maximum pair: every voxel exact
        assert err.max() <= S_TOL


def test_quaternion_maximiser_degenerate_and_rank_one(T, ctx):
    """A zero tensor gives score 0 and the identity quaternion; a rank-one
    tensor l q0^{(x)4} gives score l at +-q0 (canonical w >= 0)."""
    n, K = 4, 35
    shape = (3, 4, 40)   # no smaller than the 3^3 template on any axis
    V = int(np.prod(shape))
    a = O.multi_indices(n, 4)
    rng = np.random.default_rng(9)
    qs = rng.normal(size=(V, 4))
    qs /= np.linalg.norm(qs, axis=1, keepdims=True)
    lam = rng.uniform(0.5, 2.0, V)
    C = np.array([[lam[v] * np.prod(qs[v] ** e) for e in a] for v in range(V)]).T.copy()
    C[:, 0] = 0.0
    tmpl = synth.gaussian_blob_template(3, seed=1)
    p = T.params(order_n=n, mask_radius=1.0, n_rot_base=4, dprime=4)
    plan = T.Plan(ctx, dev(oracle_field4(tmpl, 1.0, n, 4), torch.float64), p, shape)
    s, q, F = maps(T, ctx, plan, dev(C.reshape((K,) + shape)), shape)
    s, q = s.ravel(), q.reshape(4, -1).T
    assert s[0] == 0.0 and tuple(q[0]) == (1.0, 0.0, 0.0, 0.0) and F.ravel()[0] == 0.0
    assert np.abs(s[1:] - lam[1:]).max() <= 1e-5 * lam.max()
    assert rot_angle_deg(q[1:], qs[1:]).max() <= 0.1
    assert (q[1:, 0] >= 0).all()


def test_quaternion_form_recovers_planted_rotation(T, ctx):
    """The whole d' = 4 path (GPU field, correlation, maximiser) on a noise
    tomogram with planted copies at rotations the input generator draws:
    at each centre the quaternion map gives the planted rotation (roll
    included) within 10 degrees, and C, score and rotation equal the
    oracle's (its own field, correlation and maximiser on the host copy of
    the same tomogram)."""
    N, r, n = 16, 7.0, 4
    shape = (48, 48, 48)
    tmpl = synth.gaussian_blob_template(N, seed=20240802).astype(np.float32)
    vol, pl = synth.make_tomogram(shape, tmpl, r, 3, seed=77, amplitude=5.0)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=512, dprime=4)
    m = T.Matcher(ctx, tmpl, p, shape)
    s, q, F = m.run(dev(vol))
    torch.cuda.synchronize()
    assert tuple(q.shape) == (4,) + shape
    s, q, C = s.cpu().numpy(), q.cpu().numpy(), m.C.cpu().numpy()
    field = oracle_field4(tmpl.astype(np.float64), r, n, 512)
    pr = O.Prepared(vol.astype(np.float64), tmpl.astype(np.float64), r)
    vox = np.array([(int(c[0]) * shape[1] + int(c[1])) * shape[2] + int(c[2]) for c in pl.centres])
    w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=False, floor=pr.floor)
    Cref = O.correlate(pr.g, field, vox, periodic=False, w=w)
    sref, qref, _ = O.maximise(Cref, n, 4, nsamples=20000)
    assert len(vox) >= 2
    for i, (c, q0) in enumerate(zip(pl.centres, pl.quats)):
        z, y, x = (int(v) for v in c)
        assert np.abs(C[:, z, y, x] - Cref[:, i]).max() <= C_TOL
        assert rot_angle_deg(q[:, z, y, x][None], np.asarray(q0)[None])[0] < 10.0
        assert abs(s[z, y, x] - sref[i]) <= S_TOL
        assert rot_angle_deg(q[:, z, y, x][None], qref[i][None])[0] <= ANG_TOL_DEG


def test_quaternion_unsupported_forms(T, ctx):
    tmpl = synth.gaussian_blob_template(7, seed=3)
    p = T.params(order_n=4, mask_radius=3.0, n_rot_base=4, dprime=4)
    plan = T.Plan(ctx, dev(oracle_field4(tmpl, 3.0, 4, 4), torch.float64), p, (16, 16, 16))
    d_C = torch.zeros((35, 16, 16, 16), device="cuda")
    d_s = torch.empty((16, 16, 16), device="cuda")
    d_q = torch.empty((4, 16, 16, 16), device="cuda")
    net = T.Mlp(ctx, 35, seed=1)
    with pytest.raises(T.TTMError) as e:
        T.ttm_peak_map(plan, d_C, d_s, d_q, mlp=net)
    assert e.value.code == 3
    with pytest.raises(ValueError):      # a d' = 3 sized orientation map is too small
        T.ttm_peak_map(plan, d_C, d_s, torch.empty((3, 16, 16, 16), device="cuda"))


# ------------------------------------------------------------- TTM-ref --

def test_ttm_refine_matches_oracle(T, ctx):
    """Alg. 3 on the GPU (quaternion map, real-space LNCC per candidate)
    against the oracle's TTM-ref (its own field, C, maximiser and LNCC) for
    peaks at, and 1-2 voxels off, a planted copy and one in pure noise. The
    refined voxel is unique where the oracle's best candidate leads the next
    by more than 1e-4; elsewhere the GPU's choice must be within 1e-4 of the
    oracle's best LNCC."""
    N, r, n, shape = 16, 7.0, 4, (40, 40, 40)
    tmpl = synth.gaussian_blob_template(N, seed=20240802).astype(np.float32)
    vol, pl = synth.make_tomogram(shape, tmpl, r, 1, seed=101, amplitude=5.0)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=256, dprime=4)
    m = T.Matcher(ctx, tmpl, p, shape)
    m.run(dev(vol))
    torch.cuda.synchronize()
    c = np.array(pl.centres[0], dtype=np.int64)
    Y, X = shape[1], shape[2]
    lin = lambda z, y, x: (z * Y + y) * X + x
    far = (c + np.where(c < 20, 10, -10))              # a valid voxel away from the copy
    starts = np.array([lin(*c), lin(c[0] + 1, c[1] - 1, c[2] + 2), lin(c[0] - 2, c[1], c[2]), lin(*far)])
    idx, q, val = T.ttm_refine_peaks(m.plan, dev(tmpl), m.orient, starts, 3.0)
    pr = O.Prepared(vol.astype(np.float64), tmpl.astype(np.float64), r)
    field = O.tensor_field(pr.tp, O.rotation_set(256), n, 4)
    oidx, oq, oval, cands = O.ttm_refine(pr, field, n, starts, r_s=3.0)
    for k in range(len(starts)):
        vox, cv = cands[k]
        j = np.flatnonzero(vox == idx[k])
        assert j.size == 1
        assert cv.max() - cv[j[0]] <= 1e-4
        top2 = np.sort(cv)[-2:]
        if top2[1] - top2[0] > 1e-4:
            assert idx[k] == oidx[k]
        assert abs(val[k] - cv[j[0]]) <= 1e-4
        if k < 3:
            assert idx[k] == lin(*c)
            assert rot_angle_deg(q[k][None], oq[k][None])[0] <= ANG_TOL_DEG
            assert rot_angle_deg(q[k][None], np.asarray(pl.quats[0])[None])[0] < 10.0
    # an empty list, a peak outside the valid box, and a d' = 3 plan
    assert len(T.ttm_refine_peaks(m.plan, dev(tmpl), m.orient, [], 3.0)[0]) == 0
    with pytest.raises(T.TTMError) as e:
        T.ttm_refine_peaks(m.plan, dev(tmpl), m.orient, [0], 3.0)
    assert e.value.code == 1
    p3 = T.params(order_n=2, mask_radius=r, n_rot_base=16)
    m3 = T.Matcher(ctx, tmpl, p3, shape)
    with pytest.raises(T.TTMError) as e:
        T.ttm_refine_peaks(m3.plan, dev(tmpl), m.orient, starts[:1], 3.0)
    assert e.value.code == 3


# ------------------------------------------------ synthetic accuracy study --

def test_study_noise_free_copies_recovered_exactly(T, ctx):
    """The synthetic accuracy study (the analogue of Sec. 5.1, run in full by
    bench.py --workload study), reduced to one cell: 27 copies of the 21^3
    six-Gaussian template on a 3 x 3 x 3 grid at uniform random rotations,
    noise-free, the quaternion form at n = 4 (24 x 2048 field rotations).
    The 27 highest Frobenius peaks at exclusion 2r (Sec. 3.2, 3.4) lie
    within 3 voxels of the copies (the shift Sec. 3.3 describes), and
    TTM-ref (Alg. 3, r_s = 3) puts every copy on its exact centre with the
    planted rotation to within 1 degree."""
    N, r, n = 21, 9.0, 4
    tmpl = synth.gaussian_blob_template(N, seed=11).astype(np.float32)
    vol, pl = synth.grid_tomogram(tmpl, 3, 26, 4, 31, None, r)   # 81^3
    p = T.params(order_n=n, mask_radius=r, n_rot_base=2048, dprime=4)
    m = T.Matcher(ctx, tmpl, p, vol.shape)
    m.run(dev(vol))
    torch.cuda.synchronize()
    pk, _ = T.ttm_find_peaks(m.plan, m.frob, 27, 2 * r)
    assert pk.size == 27
    Z, Y, X = vol.shape

    def zyx(i):
        i = np.asarray(i)
        return np.stack([i // (Y * X), (i // X) % Y, i % X], axis=1).astype(float)

    cen = np.asarray(pl.centres, dtype=float)
    d = np.linalg.norm(zyx(pk)[:, None, :] - cen[None, :, :], axis=2)
    assert d.min(axis=1).max() <= 3.0
    ridx, rq, _ = T.ttm_refine_peaks(m.plan, dev(tmpl), m.orient, pk, 3.0)
    d = np.linalg.norm(zyx(ridx)[:, None, :] - cen[None, :, :], axis=2)
    j = d.argmin(axis=1)
    assert d.min(axis=1).max() == 0.0
    assert sorted(j.tolist()) == list(range(27))          # every copy exactly once
    err = rot_angle_deg(rq, np.asarray(pl.quats)[j])
    assert err.max() <= 1.0, err
