"""Pins for the FP64 oracle: every check compares it with something other than
itself -- constants printed in the paper (tests/golden), closed forms,
library routines (numpy eigh), exact permutations, invariances and brute
force on tiny inputs -- so that a dropped term, a wrong sign, index or
transposed operand in the oracle fails at least one of them.
No GPU needed."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(key):
    for line in open(os.path.join(GOLDEN, "paper_constants.txt")):
        line = line.split("#", 1)[0].split()
        if len(line) == 2 and line[0] == key:
            return float(line[1])
    raise KeyError(key)


# ----------------------------------------------------------- closed forms --

def sphere_moment(alpha):
    """E[prod x_i^a_i] for x uniform on the unit sphere S^{d-1} (d = len(alpha)):
    Gamma(d/2) / Gamma((n+d)/2) * prod Gamma((a_i+1)/2) / Gamma(1/2), zero if
    any exponent is odd."""
    d = len(alpha)
    n = sum(alpha)
    if any(a % 2 for a in alpha):
        return 0.0
    v = math.gamma(d / 2) / math.gamma((n + d) / 2)
    for a in alpha:
        v *= math.gamma((a + 1) / 2) / math.gamma(0.5)
    return v


def full_tensor(c, n, d):
    """Expand independent components into the full symmetric d^n tensor (each
    entry takes the value of the component of its sorted index multiset)."""
    idx = O.multi_indices(n, d)
    lookup = {tuple(a): k for k, a in enumerate(idx)}
    T = np.zeros((d,) * n)
    for ent in itertools.product(range(d), repeat=n):
        cnt = tuple(ent.count(i) for i in range(d))
        T[ent] = c[lookup[cnt]]
    return T


def contract(T, u, times):
    for _ in range(times):
        T = T @ u
    return T


def cube_matrices():
    """The 24 proper rotations of the cube, as signed permutation matrices
    with determinant +1 (built here independently of the oracle)."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3))
            for r, (c, s) in enumerate(zip(perm, signs)):
                P[r, c] = s
            if round(np.linalg.det(P)) == 1:
                mats.append(P)
    return mats


def centred_grid(N):
    c = N // 2
    g = np.arange(N) - c
    pz, py, px = np.meshgrid(g, g, g, indexing="ij")
    return px, py, pz


def permute_by(t, P):
    """out(p) = t(P^T p) on an odd cubic grid (exact voxel permutation)."""
    N = t.shape[0]
    c = N // 2
    px, py, pz = centred_grid(N)
    Pv = np.stack([px.ravel(), py.ravel(), pz.ravel()])
    src = (P.T @ Pv).round().astype(int) + c
    return t[src[2], src[1], src[0]].reshape(t.shape)


# ------------------------------------------------------------ index sets --

def test_component_counts_match_paper():
    # Sec. 3 after Alg. 2: n = 4 with quaternions (d' = 4) needs 35 correlations
    assert O.num_components(4, 4) == int(golden("components_n4_d4"))
    for n in (2, 4, 6):
        assert O.num_components(n, 3) == (n + 1) * (n + 2) // 2
    assert [O.num_components(n, 3) for n in (2, 4, 6)] == [6, 15, 28]


@pytest.mark.parametrize("n,d", [(2, 3), (4, 3), (6, 3), (2, 4), (4, 4), (6, 4)])
def test_multi_indices_enumerate_all_multisets(n, d):
    a = O.multi_indices(n, d)
    brute = {tuple(sum(1 for e in comb if e == i) for i in range(d))
             for comb in itertools.combinations_with_replacement(range(d), n)}
    assert set(map(tuple, a)) == brute
    assert len(a) == len(brute)
    # graded-lex descending: first exponents non-increasing lexicographically
    assert [tuple(x) for x in a] == sorted(map(tuple, a), reverse=True)
    # multiplicities count the full-tensor entries: they sum to d^n
    m = O.multiplicities(n, d)
    assert m.sum() == pytest.approx(d ** n)


@pytest.mark.parametrize("n,d", [(2, 3), (4, 3), (6, 3), (4, 4), (6, 4)])
def test_frobenius_of_tensor_power(n, d):
    rng = np.random.default_rng(1)
    v = rng.normal(size=d)
    a = O.multi_indices(n, d)
    c = np.array([np.prod(v ** e) for e in a])  # components of v^{(x)n}
    F = O.frobenius(c[:, None], n, d)[0]
    assert F == pytest.approx(np.linalg.norm(v) ** n, rel=1e-12)
    assert F == pytest.approx(np.linalg.norm(full_tensor(c, n, d)), rel=1e-12)


# -------------------------------------------------------------- filter h --

def test_filter_taps_and_response():
    a = golden("filter_a")
    assert 0 < a < golden("filter_a_upper")
    f = np.zeros((5, 5, 5))
    f[2, 2, 2] = 1.0
    g = O.filter3(f, a)
    taps = np.array([a, 1 - 2 * a, a])  # z-transform 1 + a(z + 1/z - 2)
    assert np.allclose(g[1:4, 1:4, 1:4], np.einsum("i,j,k->ijk", taps, taps, taps), atol=1e-15)
    assert g.sum() == pytest.approx(1.0)
    # constant interior is preserved; zero padding loses one tap per touched edge
    g1 = O.filter3(np.ones((6, 6, 6)), a)
    assert np.allclose(g1[1:-1, 1:-1, 1:-1], 1.0)
    assert g1[0, 0, 0] == pytest.approx((1 - a) ** 3)
    # Nyquist along x: H(z = -1) = 1 - 4a
    x = np.arange(8)
    alt = np.broadcast_to((-1.0) ** x, (8, 8, 8)).copy()
    ga = O.filter3(alt, a)
    assert np.allclose(ga[1:-1, 1:-1, 1:-1], (1 - 4 * a) * alt[1:-1, 1:-1, 1:-1])


# ------------------------------------------------------------------ mask --

def test_mask_count_and_soft_edge():
    m, M = O.mask((16, 16, 16), 7.0)
    px, py, pz = centred_grid(16)
    brute = int(np.sum(px ** 2 + py ** 2 + pz ** 2 <= 49))
    assert M == brute == int(m.sum())
    assert set(np.unique(m)) <= {0.0, 1.0}
    ms, Ms = O.mask((21, 21, 21), 6.0, soft=2.0)
    rho = np.sqrt(np.add.reduce([c.astype(float) ** 2 for c in centred_grid(21)]))
    assert np.all(ms[rho <= 6] == 1.0)
    assert np.all(ms[rho >= 8] == 0.0)
    ramp = (rho > 6) & (rho < 8)
    assert np.all((ms[ramp] > 0) & (ms[ramp] < 1))
    order = np.argsort(rho[ramp])
    assert np.all(np.diff(ms[ramp][order]) <= 1e-15)


# ------------------------------------------------- template normalisation --

def test_template_normalisation_eq4():
    t = synth.gaussian_blob_template(15, seed=7)
    m, M = O.mask(t.shape, 6.0)
    tp, den = O.normalise_template(t, m)
    assert np.all(tp[m == 0] == 0)
    assert tp.sum() == pytest.approx(0.0, abs=1e-12)          # zero mean under the mask
    assert (tp ** 2).sum() == pytest.approx(1.0, rel=1e-12)   # unit norm
    # invariant to affine intensity changes (mask is 1+ voxel from the grid edge)
    tp2, _ = O.normalise_template(3.5 * t - 2.0, m)
    assert np.allclose(tp, tp2, atol=1e-12)


# ------------------------------------------------------------- rotations --

def test_superfib_constants_and_moments():
    psi = O.superfib_psi()
    assert psi ** 4 == pytest.approx(psi + 4, rel=1e-15)
    q = O.superfib(4096)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)
    # low-order moments of uniform S^3 points (the SO(3) Haar measure)
    for alpha in [(2, 0, 0, 0), (0, 0, 2, 0), (1, 1, 0, 0), (4, 0, 0, 0), (2, 2, 0, 0),
                  (0, 2, 0, 2)]:
        est = np.mean(np.prod(q ** np.array(alpha), axis=1))
        assert est == pytest.approx(sphere_moment(alpha), abs=2e-3)


def test_quaternion_conventions():
    rng = np.random.default_rng(3)
    for _ in range(5):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        R = O.quat_to_rot(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0)
        # Rodrigues' formula for the same axis-angle
        ang = 2 * math.acos(max(-1.0, min(1.0, q[0])))
        ax = q[1:] / np.linalg.norm(q[1:])
        Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        Rr = np.eye(3) + math.sin(ang) * Kx + (1 - math.cos(ang)) * Kx @ Kx
        assert np.allclose(R, Rr, atol=1e-12)
    # rot(p q) = rot(p) rot(q)
    p = np.array([0.5, 0.5, 0.5, 0.5])
    q = np.array([math.cos(0.3), 0, math.sin(0.3), 0])
    assert np.allclose(O.quat_to_rot(O.quat_mul(p, q)), O.quat_to_rot(p) @ O.quat_to_rot(q))


def test_cube_group_is_the_cube_group():
    qs = O.cube_rotations()
    mats = [O.quat_to_rot(q) for q in qs]
    ref = cube_matrices()
    assert len(ref) == 24
    for R in mats:
        assert np.allclose(R, np.round(R), atol=1e-12)
    key = lambda R: tuple(np.round(R).astype(int).ravel())
    assert {key(R) for R in mats} == {key(P) for P in ref}


def test_rotate_template_exact_for_cube_rotations():
    t = synth.gaussian_blob_template(13, seed=11)
    for q in O.cube_rotations():
        R = O.quat_to_rot(q)
        assert np.allclose(O.rotate_template(t, q), permute_by(t, np.round(R)), atol=1e-14)
    # quarter-turn about z maps the +x axis onto +y: a blob at +x moves to +y
    t = np.zeros((9, 9, 9))
    t[4, 4, 7] = 1.0                       # (x,y,z) offset (3,0,0)
    q90z = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    r = O.rotate_template(t, q90z)
    assert r[4, 7, 4] == pytest.approx(1.0)  # offset (0,3,0)


# ---------------------------------------------------------- tensor field --

@pytest.mark.parametrize("n", [2, 4])
def test_field_exact_under_cube_quadrature(n):
    """Alg. 1 with Q = the 24 cube rotations and an odd template: every
    resampling is an exact voxel permutation, so T_alpha(p) =
    (1/24) sum_P (P e_z)^alpha t'(P^T p) can be written out exactly."""
    t = synth.gaussian_blob_template(11, seed=5)
    m, _ = O.mask(t.shape, 4.0)
    tp, _ = O.normalise_template(t, m)
    T = O.tensor_field(tp, O.cube_rotations(), n, 3)
    alpha = O.multi_indices(n, 3)
    ref = np.zeros_like(T)
    for P in cube_matrices():
        u = P[:, 2]
        rot = permute_by(tp, P)
        for k, a in enumerate(alpha):
            ref[k] += np.prod(u ** a) * rot
    ref /= 24.0
    assert np.abs(T - ref).max() < 1e-14


@pytest.mark.parametrize("n,d", [(2, 3), (4, 3), (6, 3), (2, 4), (4, 4), (6, 4)])
def test_field_of_constant_is_sphere_moment(n, d):
    """A constant t' is reproduced exactly by trilinear resampling away from
    the grid edge, so T_alpha there equals the quadrature of E[u^alpha] over
    S^2 (u = R e_z) or S^3 (u = q): a closed form."""
    N = 9
    tp = np.ones((N, N, N))
    Q = O.rotation_set(256, cube=True)
    T = O.tensor_field(tp, Q, n, d)
    alpha = O.multi_indices(n, d)
    ctr = T[:, N // 2, N // 2, N // 2]
    ref = np.array([sphere_moment(tuple(a)) for a in alpha])
    assert np.abs(ctr - ref).max() < 2e-3
    # one voxel off-centre, still fully inside after any rotation
    assert np.abs(T[:, N // 2 + 1, N // 2, N // 2 - 1] - ref).max() < 2e-3


def test_field_quadrature_converges():
    """Doubling the super-Fibonacci quadrature of Eq. 9 shrinks the change in T.
    Trilinear resampling makes the integrand only continuous in R, so the
    rate is slow: about 1e-3 relative at the default 24 x 2048 rotations."""
    t = synth.gaussian_blob_template(16, seed=20240802)
    m, _ = O.mask(t.shape, 7.0)
    tp, _ = O.normalise_template(t, m)
    T = {nb: O.tensor_field(tp, O.rotation_set(nb), 2, 3) for nb in (128, 256, 1024, 2048)}
    scale = np.abs(T[2048]).max()
    coarse = np.abs(T[256] - T[128]).max() / scale
    fine = np.abs(T[2048] - T[1024]).max() / scale
    assert fine < 0.25 * coarse
    assert fine < 3e-3


# ------------------------------------------------------ local normaliser --

def test_local_w_linear_ramp_closed_form():
    """g(x) = beta * x_x: S1 = beta M x, S2 = beta^2 (M x^2 + sum_ball p_x^2),
    so var = beta^2 sum_{p in ball} p_x^2 exactly."""
    Z = Y = X = 24
    beta = 0.37
    g = np.broadcast_to(beta * np.arange(X, dtype=float), (Z, Y, X)).copy()
    m, M = O.mask((11, 11, 11), 4.0)
    px, py, pz = centred_grid(11)
    sum_px2 = float(np.sum(px[m > 0] ** 2))
    vox = O.valid_voxels(g.shape, m.shape)[::97]
    w, S1, S2 = O.local_w(g, m, vox)
    xs = vox % X
    assert np.allclose(S1, beta * M * xs, rtol=1e-12)
    assert np.allclose(w, 1.0 / (beta * math.sqrt(sum_px2)), rtol=1e-10)
    # constant image: zero variance -> w = 0 by the floor rule
    wc, _, _ = O.local_w(np.full((Z, Y, X), 3.0), m, vox, floor=1e-12)
    assert np.all(wc == 0)


def test_local_w_zero_variance_floor_counts_sliver_windows():
    """The zero-variance floor of the normaliser (w = 0 where the local
    variance is at most 1e-8 M mean(g^2)), on windows that hold only a
    sliver of an object in an exactly empty background.

    Volume: zeros, a block of ones far away (it sets mean(g^2)) and a single
    voxel of value v at c0. The mask is the radius-1 ball (centre and its 6
    face neighbours, M = 7). After the 3-tap filter (0.2, 0.6, 0.2 per axis)
    the single voxel becomes a 3x3x3 cube of products of taps: 0.216 v at
    c0, 0.072 v on faces, 0.024 v on edges, 0.008 v on corners. By hand:
      - windows that touch that cube are the cube dilated by the 6-neighbour
        ball: 27 + 6 * 9 = 81 voxels;
      - the window at c0 sees 0.216 v and six 0.072 v: S1 = 0.648 v,
        S2 = 0.07776 v^2, var = S2 - S1^2 / 7 = 0.0177737... v^2 (the
        largest of the 81);
      - the window at c0 + (2, 1, 1) sees one corner only: var = 0.008^2
        (1 - 1/7) v^2 = 5.4857e-5 v^2 (the smallest, 324 times less).
    v is chosen so that the largest sliver variance is 1e-9 M mean(g^2):
    all 81 lie between the two floors, so exactly 81 voxels have w = 0 at
    1e-8 but w > 0 at 1e-12 (block-interior and empty windows have zero
    variance, block-edge windows variance far above both floors)."""
    Z = Y = X = 26
    f = np.zeros((Z, Y, X))
    f[15:23, 15:23, 15:23] = 1.0
    m, M = O.mask((3, 3, 3), 1.0)
    assert M == 7
    c0 = (6, 7, 8)
    g_block = O.filter3(f)
    E_block = M * float(np.mean(g_block ** 2))
    var_max_unit = 0.07776 - 0.648 ** 2 / 7.0
    v = math.sqrt(1e-9 * E_block / var_max_unit)
    f[c0] = v
    g = O.filter3(f)
    E = M * float(np.mean(g ** 2))
    vox = O.valid_voxels(g.shape, m.shape)
    w8, _, _ = O.local_w(g, m, vox, floor=1e-8 * E)
    w12, _, _ = O.local_w(g, m, vox, floor=1e-12 * E)
    wd, _, _ = O.local_w(g, m, vox)          # the default floor is the 1e-8 one
    assert np.array_equal(wd, w8)
    sliver = (w8 == 0) & (w12 > 0)
    assert int(sliver.sum()) == 81
    zz, yy, xx = np.unravel_index(vox[sliver], g.shape)
    d = np.abs(np.stack([zz, yy, xx], 1) - np.array(c0))
    # inside the dilated cube: at most 2 per axis and at most one axis at 2
    assert np.all(d.max(1) <= 2) and np.all((d == 2).sum(1) <= 1)
    at = {tuple(p): k for k, p in enumerate(np.stack([zz, yy, xx], 1))}
    k_c = at[c0]
    k_corner = at[(c0[0] + 2, c0[1] + 1, c0[2] + 1)]
    assert w12[sliver][k_c] == pytest.approx(1.0 / math.sqrt(var_max_unit * v * v), rel=1e-9)
    assert w12[sliver][k_corner] == pytest.approx(1.0 / math.sqrt(0.008 ** 2 * (6.0 / 7.0) * v * v), rel=1e-9)


def test_local_w_periodic_agrees_in_interior():
    g = synth.normals(9, 1, 20 ** 3).reshape(20, 20, 20)
    m, _ = O.mask((7, 7, 7), 3.0)
    vox = O.valid_voxels(g.shape, m.shape)
    w0, _, _ = O.local_w(g, m, vox, periodic=False, floor=0.0)
    w1, _, _ = O.local_w(g, m, vox, periodic=True, floor=0.0)
    assert np.array_equal(w0, w1)


# ----------------------------------------------------------- correlation --

def test_correlation_of_delta_is_reflected_template():
    """Eq. 5: (g * T)(x) = sum_p g(x+p) T(p); for g = delta at x0 this is
    T(x0 - x) (correlation, not convolution)."""
    Z = Y = X = 12
    T = synth.gaussian_blob_template(5, seed=3)[None]
    g = np.zeros((Z, Y, X))
    x0 = (6, 5, 7)
    g[x0] = 1.0
    out = O.correlate(g, T, periodic=False)[0].reshape(Z, Y, X)
    for x in [(6, 5, 7), (5, 5, 7), (6, 4, 8), (7, 6, 6), (4, 3, 5)]:
        p = tuple(a - b for a, b in zip(x0, x))
        expect = T[0][tuple(pi + 2 for pi in p)] if all(-2 <= pi <= 2 for pi in p) else 0.0
        assert out[x] == pytest.approx(expect, abs=1e-15)


def test_lncc_is_one_at_a_perfect_match():
    """Eqs. 1-5: a tomogram holding an exact copy of the template (any
    positive gain and offset) gives LNCC 1 at the copy's centre."""
    N = 13
    t = synth.gaussian_blob_template(N, seed=13)
    m, M = O.mask(t.shape, 5.0)
    tp, _ = O.normalise_template(t, m)
    Z = Y = X = 32
    f = np.zeros((Z, Y, X))
    c0 = (15, 17, 14)
    h = N // 2
    f[c0[0] - h:c0[0] - h + N, c0[1] - h:c0[1] - h + N, c0[2] - h:c0[2] - h + N] = t
    for gain, off in [(1.0, 0.0), (2.5, -0.7)]:
        g = O.filter3(gain * f + off)
        v = np.array([(c0[0] * Y + c0[1]) * X + c0[2]])
        w, _, _ = O.local_w(g, m, v)
        c = O.correlate(g, tp[None], v, w=w)[0, 0]
        assert c == pytest.approx(1.0, abs=1e-12)


def test_lncc_bounded_by_one_and_scale_invariant():
    g = O.filter3(synth.normals(4, 1, 18 ** 3).reshape(18, 18, 18))
    t = synth.gaussian_blob_template(7, seed=4)
    m, _ = O.mask(t.shape, 3.0)
    tp, _ = O.normalise_template(t, m)
    vox = O.valid_voxels(g.shape, t.shape)
    best, _ = O.tm(g, tp, O.cube_rotations(), vox, w=O.local_w(g, m, vox)[0])
    assert np.all(np.abs(best) <= 1 + 1e-12)
    best2, _ = O.tm(4.0 * g, tp, O.cube_rotations(), vox, w=O.local_w(4.0 * g, m, vox)[0])
    assert np.allclose(best, best2, atol=1e-12)


def test_tm_recovers_planted_quarter_turn():
    """A copy rotated by a quarter-turn about z is found with LNCC 1 at that
    rotation's index -- and not at the inverse quarter-turn."""
    N = 11
    t = synth.gaussian_blob_template(N, seed=21)
    m, _ = O.mask(t.shape, 4.0)
    tp, _ = O.normalise_template(t, m)
    s = math.sqrt(0.5)
    quats = np.array([[1, 0, 0, 0], [s, 0, 0, s], [s, 0, 0, -s], [0, 0, 0, 1.0]])
    R = O.quat_to_rot(quats[1])
    Z = Y = X = 27
    f = np.zeros((Z, Y, X))
    c0 = (13, 13, 13)
    h = N // 2
    f[c0[0] - h:c0[0] + h + 1, c0[1] - h:c0[1] + h + 1, c0[2] - h:c0[2] + h + 1] = permute_by(t, np.round(R))
    g = O.filter3(f)
    v = np.array([(c0[0] * Y + c0[1]) * X + c0[2]])
    w, _, _ = O.local_w(g, m, v)
    best, idx = O.tm(g, tp, quats, v, w=w)
    assert idx[0] == 1
    assert best[0] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.slow
def test_brute_force_tm_agrees_with_ttm_ref_on_planted_copies():
    """Classical TM at fine angular sampling (Eqs. 1, 6, 7 over 100 008
    super-Fibonacci rotations, cube-symmetrised) against TTM on a tiny
    volume: a 20 x 20 x 22 tomogram with two copies of a compact 9^3
    four-Gaussian template, planted at rotations taken from the TM list
    (so TM's answer at the copies is defined: that index), light white
    noise (sigma 0.02). Over the whole valid interior:
      - TM's two highest peaks (exclusion 2 r) are the planted centres, and
        its best rotation there is the planted one;
      - TTM's score peaks (d' = 4, n = 4, Sec. 3.1) lie within r_s = 3
        voxels of them (Sec. 3.3: TTM peaks may be shifted);
      - TTM-ref (Alg. 3, r_s = 3) moves them exactly onto TM's peaks, with
        rotations within 3 degrees of TM's.
    The d' = 3 axis u* against TM's best R e_z is printed, not gated."""
    N, r = 9, 4.0
    tmpl = synth.gaussian_blob_template(N, seed=7, n_blobs=4, centre_radius=2.5, std_lo=0.7, std_hi=1.6)
    shape = (20, 20, 22)
    Q = O.rotation_set(4167, cube=True)
    assert Q.shape[0] >= 100000
    planted_idx = [31337, 77777]
    cen = np.array([[7, 7, 7], [13, 12, 14]])
    vol = np.zeros(shape)
    synth.plant(vol, tmpl, cen, Q[planted_idx], 1.0)
    vol += 0.02 * synth.normals(98, 1, vol.size).reshape(shape)
    pr = O.Prepared(vol, tmpl, r)
    vox = O.valid_voxels(shape, tmpl.shape)
    Z, Y, X = shape
    box = (N // 2, Z - (N - N // 2) + 1, N // 2, Y - (N - N // 2) + 1, N // 2, X - (N - N // 2) + 1)
    w, _, _ = O.local_w(pr.g, pr.m, vox, False, pr.floor)
    best, bidx = O.tm(pr.g, pr.tp, Q, vox, False, w)
    full = np.full(Z * Y * X, -np.inf)
    full[vox] = best
    tm_pk, tm_val = O.find_peaks(full.reshape(shape), box, 2, 2 * r)
    cen_idx = (cen[:, 0] * Y + cen[:, 1]) * X + cen[:, 2]
    assert set(tm_pk.tolist()) == set(cen_idx.tolist())
    pos = {int(v): k for k, v in enumerate(vox)}
    for c, qi in zip(cen_idx, planted_idx):
        assert bidx[pos[int(c)]] == qi
    # TTM, the paper's quaternion form
    F4 = O.tensor_field(pr.tp, O.rotation_set(512), 4, 4)
    C = O.correlate(pr.g, F4, vox, False, w)
    s4, _, _ = O.maximise(C, 4, 4, 20000)
    full = np.full(Z * Y * X, -np.inf)
    full[vox] = s4
    ttm_pk, _ = O.find_peaks(full.reshape(shape), box, 2, 2 * r)

    def zyx(i):
        return np.array([i // (Y * X), (i // X) % Y, i % X], dtype=float)
    for c in cen_idx:
        assert min(np.linalg.norm(zyx(c) - zyx(p)) for p in ttm_pk) <= 3.0
    ref_pk, ref_q, _, _ = O.ttm_refine(pr, F4, 4, ttm_pk, 3.0)
    assert set(ref_pk.tolist()) == set(tm_pk.tolist())
    for p, q in zip(ref_pk, ref_q):
        q_tm = Q[bidx[pos[int(p)]]]
        assert math.degrees(2 * math.acos(min(1.0, abs(float(np.dot(q, q_tm)))))) <= 3.0
    # reported: the d' = 3 needle axis against TM's best R e_z
    F3 = O.tensor_field(pr.tp, O.rotation_set(512), 4, 3)
    for c in cen_idx:
        k = pos[int(c)]
        _, u3, _ = O.maximise(O.correlate(pr.g, F3, vox[k:k + 1], False, w[k:k + 1]), 4, 3, 20000)
        ez = O.quat_to_rot(Q[bidx[k]])[:, 2]
        print("d'=3 u* vs TM R e_z at %s: %.1f deg" % (tuple(int(t) for t in zyx(c)),
                                                     math.degrees(math.acos(min(1.0, abs(float(u3[0] @ ez)))))))


# ------------------------------------------------------------- maximiser --

def test_maximiser_order2_is_top_eigenpair():
    C = synth.random_tensors(17, 40, 6).T.copy()   # [K][nvox]
    s, u, _ = O.maximise(C, 2, 3, nsamples=2000)
    for i in range(C.shape[1]):
        c = C[:, i]
        A = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        ev, V = np.linalg.eigh(A)
        assert s[i] == pytest.approx(ev[-1], abs=1e-12)
        assert abs(abs(u[i] @ V[:, -1]) - 1) < 1e-10


def test_quaternion_order2_is_top_eigenpair():
    """d' = 4, n = 2: p(q) = q^T A q with A_ij = C_{e_i + e_j} (4 x 4), so
    the maximum over unit quaternions is the top eigenpair of A; the
    canonical quaternion has its first non-zero entry (w) positive."""
    idx = {tuple(a): k for k, a in enumerate(O.multi_indices(2, 4))}
    C = synth.random_tensors(18, 40, 10).T.copy()
    s, u, _ = O.maximise(C, 2, 4, nsamples=4000)
    for i in range(C.shape[1]):
        A = np.empty((4, 4))
        for a in range(4):
            for b in range(4):
                e = [0, 0, 0, 0]
                e[a] += 1
                e[b] += 1
                A[a, b] = C[idx[tuple(e)], i]
        ev, V = np.linalg.eigh(A)
        assert s[i] == pytest.approx(ev[-1], abs=1e-12)
        assert abs(abs(u[i] @ V[:, -1]) - 1) < 1e-10
        assert u[i][0] > 0


def test_quaternion_rank_one_and_two():
    """d' = 4, n = 4: C = l1 q1^{(x)4} + l2 q2^{(x)4} with orthogonal unit
    quaternions has its maximum l1 at +-q1."""
    rng = np.random.default_rng(44)
    a = O.multi_indices(4, 4)
    for _ in range(5):
        Qm, _ = np.linalg.qr(rng.normal(size=(4, 4)))
        q1, q2 = Qm[:, 0], Qm[:, 1]
        c = np.array([2.0 * np.prod(q1 ** e) + 1.3 * np.prod(q2 ** e) for e in a])
        s, u, _ = O.maximise(c[:, None], 4, 4, nsamples=8000)
        assert s[0] == pytest.approx(2.0, abs=1e-12)
        assert abs(abs(u[0] @ q1) - 1) < 1e-10


@pytest.mark.parametrize("n", [2, 4])
def test_quaternion_form_recovers_planted_rotation(n):
    """Sec. 3: with d' = 4 the maximising quaternion is the full rotation
    (roll included) of a planted copy. The copies are placed by the input
    generator's own resampler at rotations it draws (not by the oracle);
    the order-n smoothing of Eq. 9 biases the maximum by a few degrees, so
    the bound is 10 degrees."""
    N, r, shape = 16, 7.0, (40, 40, 40)
    tmpl = synth.gaussian_blob_template(N, seed=20240802)
    m, _ = O.mask(tmpl.shape, r)
    tp, _ = O.normalise_template(tmpl, m)
    field = O.tensor_field(tp, O.rotation_set(512), n, 4)
    for seed in range(3):
        vol, pl = synth.make_tomogram(shape, tmpl, r, 1, seed=100 + seed, amplitude=5.0)
        c = pl.centres[0]
        pr = O.Prepared(vol.astype(np.float64), tmpl, r)
        v = np.array([(c[0] * shape[1] + c[1]) * shape[2] + c[2]])
        w, _, _ = O.local_w(pr.g, pr.m, v, periodic=False, floor=pr.floor)
        C = O.correlate(pr.g, field, v, periodic=False, w=w)
        s, u, _ = O.maximise(C, n, 4, nsamples=20000)
        R0, R1 = O.quat_to_rot(pl.quats[0]), O.quat_to_rot(u[0])
        ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R0.T @ R1) - 1) / 2))))
        assert ang < 10.0, (seed, ang)
        assert s[0] > 0


def test_ttm_refine_moves_shifted_peak_to_planted_centre():
    """Alg. 3: a peak placed 1-2 voxels off a planted copy moves back to the
    copy's centre (placed by the input generator, not the oracle), with the
    copy's rotation, and the LNCC there exceeds the LNCC at the shifted
    start. The candidate set is the ball of radius 3 (123 voxels) in
    (z, y, x) order after the peak itself."""
    offs = O.ball_offsets(3.0)
    assert len(offs) == 123 and tuple(offs[0]) == (0, 0, 0)
    assert (np.sum(offs ** 2, axis=1) <= 9).all()
    assert [tuple(o) for o in offs[1:]] == sorted(tuple(o) for o in offs[1:])
    N, r, n, shape = 16, 7.0, 4, (40, 40, 40)
    tmpl = synth.gaussian_blob_template(N, seed=20240802)
    vol, pl = synth.make_tomogram(shape, tmpl, r, 1, seed=101, amplitude=5.0)
    pr = O.Prepared(vol.astype(np.float64), tmpl, r)
    field = O.tensor_field(pr.tp, O.rotation_set(256), n, 4)
    c = np.array(pl.centres[0], dtype=np.int64)
    Y, X = shape[1], shape[2]
    true = (c[0] * Y + c[1]) * X + c[2]
    starts = [true, ((c[0] + 1) * Y + c[1] - 1) * X + c[2] + 2, ((c[0] - 2) * Y + c[1]) * X + c[2]]
    idx, q, val, cands = O.ttm_refine(pr, field, n, starts, r_s=3.0, nsamples=8000)
    assert (idx == true).all()
    for k in range(3):
        R0, R1 = O.quat_to_rot(pl.quats[0]), O.quat_to_rot(q[k])
        ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R0.T @ R1) - 1) / 2))))
        assert ang < 10.0
        vox, cv = cands[k]
        assert val[k] == cv.max()
        if k > 0:
            assert val[k] > cv[0] + 0.05          # better than at the shifted start
    assert val[0] > 0.9                            # the copy dominates its window (amplitude 5)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_maximiser_rank_one_and_two(n):
    rng = np.random.default_rng(n)
    a = O.multi_indices(n, 3)
    for _ in range(5):
        Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        v1, v2 = Qm[:, 0], Qm[:, 1]
        l1, l2 = 2.0, 1.3
        c = np.array([l1 * np.prod(v1 ** e) + l2 * np.prod(v2 ** e) for e in a])
        s, u, _ = O.maximise(c[:, None], n, 3, nsamples=4000)
        assert s[0] == pytest.approx(l1, abs=1e-12)
        assert abs(abs(u[0] @ v1) - 1) < 1e-10
        assert u[0][2] >= 0  # canonical half-sphere


@pytest.mark.parametrize("n,d", [(4, 3), (6, 3), (4, 4)])
def test_maximiser_random_tensors_against_full_tensor(n, d):
    K = O.num_components(n, d)
    C = synth.random_tensors(100 + n + d, 12, K).T.copy()
    s, u, _ = O.maximise(C, n, d, nsamples=20000)
    F = O.frobenius(C, n, d)
    rng = np.random.default_rng(5)
    dirs = rng.normal(size=(100000, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for i in range(C.shape[1]):
        T = full_tensor(C[:, i], n, d)
        ui = u[i]
        # the oracle's polynomial is the tensor's form: p(u) = T . u^n
        assert O.poly_eval(C[:, i], n, d, ui)[0] == pytest.approx(contract(T, ui, n), abs=1e-12)
        # Z-eigenpair: T u^{n-1} = s u
        assert np.linalg.norm(contract(T, ui, n - 1) - s[i] * ui) < 1e-10
        # Riemannian Hessian negative semidefinite at the maximum
        H = n * (n - 1) * contract(T, ui, n - 2)
        Pm = np.eye(d) - np.outer(ui, ui)
        Hr = Pm @ H @ Pm - n * s[i] * Pm
        assert np.linalg.eigvalsh(Hr).max() < 1e-8
        # s <= ||T||_F, and no random direction beats it
        assert s[i] <= F[i] + 1e-12
        brute = batch_form(T, dirs, n)
        assert brute.max() <= s[i] + 1e-12
        assert s[i] - brute.max() < 5e-3 * F[i]
        # the sphere mean bounds the max from below
        assert s[i] >= brute.mean() - 1e-12


def batch_form(T, U, n):
    """T . u^n for every row u of U (contract all n axes)."""
    vals = np.empty(U.shape[0])
    for j in range(0, U.shape[0], 5000):
        blk = U[j:j + 5000]
        R = np.tensordot(blk, T, axes=([1], [0]))        # (b, d, ..., d)
        for _ in range(n - 1):
            R = np.einsum("bi,bi...->b...", blk, R)
        vals[j:j + 5000] = R
    return vals



def test_spectral_bound_reported():
    """Sec. 3.2 quotes ||T||_sigma >= ||T||_F / 2^{n-1}; log the worst ratio
    seen on random tensors (informational, not a gate)."""
    n = 4
    C = synth.random_tensors(77, 50, 15).T.copy()
    s, _, _ = O.maximise(C, n, 3, nsamples=4000)
    F = O.frobenius(C, n, 3)
    # spectral norm = max |p| = max(max p, -min p); max p alone already bounds it below
    ratio = (np.abs(s) / F).min()
    assert ratio > 0


# ---------------------------------------------------------------- peaks --

def test_find_peaks_order_exclusion_and_ties():
    s = np.zeros((10, 10, 10))
    s[2, 2, 2] = 5.0
    s[2, 2, 5] = 4.0      # 3 voxels from the first: excluded at min_dist 4
    s[7, 7, 7] = 3.0
    s[7, 7, 3] = 3.0      # tie with (7,7,7): lower linear index first
    s[2, 8, 8] = 1.0      # >= 4 from every accepted peak
    box = (0, 10, 0, 10, 0, 10)
    idx, val = O.find_peaks(s, box, 10, 4.0)
    lin = lambda z, y, x: (z * 10 + y) * 10 + x
    assert list(idx) == [lin(2, 2, 2), lin(7, 7, 3), lin(7, 7, 7), lin(2, 8, 8)]
    assert list(val) == [5.0, 3.0, 3.0, 1.0]
    idx2, _ = O.find_peaks(s, box, 2, 4.0)
    assert list(idx2) == [lin(2, 2, 2), lin(7, 7, 3)]
    # each plateau yields one peak, at its lowest linear index (the zero
    # background is a plateau too)
    p = np.zeros((6, 6, 6))
    p[2:4, 2:4, 2:4] = 1.0
    idx3, _ = O.find_peaks(p, (0, 6, 0, 6, 0, 6), 5, 1.0)
    assert list(idx3) == [lin6(2, 2, 2), 0]


def lin6(z, y, x):
    return (z * 6 + y) * 6 + x


# ------------------------------------------------------ end-to-end pins --

@pytest.mark.slow
def test_ttm_invariant_under_quarter_turns_of_the_tomogram():
    """With a cube-symmetrised quadrature and an odd template, rotating a
    cubic tomogram by a quarter-turn rotates the score map with it and the
    orientation by the same rotation (exact up to rounding)."""
    L, N = 21, 7
    tomo = synth.normals(31, 1, L ** 3).reshape(L, L, L)
    tmpl = synth.gaussian_blob_template(N, seed=31)
    Q = O.rotation_set(64, cube=True)
    vox = O.valid_voxels((L, L, L), (N, N, N))
    base = O.ttm(tomo, tmpl, 3.0, 4, Q, vox, nsamples=3000)
    # quarter-turn about z (x -> y): array axes (z, y, x), rotate in the (y, x) plane
    P = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])   # acting on (x, y, z)
    rot = permute_by(tomo, P)
    moved = O.ttm(rot, tmpl, 3.0, 4, Q, vox, nsamples=3000)
    s0 = base["score"].reshape(-1)
    # voxel x (offset p from the volume centre) maps to P p
    c = L // 2
    zz, yy, xx = np.unravel_index(vox, (L, L, L))
    pv = np.stack([xx - c, yy - c, zz - c])
    q = (P @ pv).round().astype(int) + c
    vmap = (q[2] * L + q[1]) * L + q[0]
    pos = {v: i for i, v in enumerate(vox)}
    j = np.array([pos[v] for v in vmap])
    assert np.abs(moved["score"][j] - s0).max() < 1e-10
    ok = (base["score"] - base["second"]) > 1e-3 * np.abs(base["score"])
    u0 = base["orient"] @ P.T
    dots = np.abs(np.sum(u0[ok] * moved["orient"][j][ok], axis=1))
    assert np.all(dots > 1 - 1e-9)


# -------------------------------------------------------- learned start --

def test_mlp_gradient_matches_finite_differences():
    """Backward pass of the MLP reference against central differences of its
    own loss (relative 1e-6)."""
    K, H = 7, 9
    rng = np.random.default_rng(11)
    P = rng.normal(size=O.mlp_num_params(K, H)) * 0.6
    X = rng.normal(size=(6, K))
    U = rng.normal(size=(6, 3))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    _, L, g = O.mlp(P, X, U, H=H, want_grad=True)
    eps = 1e-6
    fd = np.empty_like(g)
    for i in range(P.size):
        e = np.zeros_like(P)
        e[i] = eps
        fd[i] = (O.mlp(P + e, X, U, H=H)[1] - O.mlp(P - e, X, U, H=H)[1]) / (2 * eps)
    assert np.abs(fd - g).max() <= 1e-6 * max(1.0, np.abs(g).max())


def test_mlp_closed_form_and_sign_invariance():
    """One hidden unit: y = (GELU(GELU(x)), 0, 0) + (0, 1, 0), so
    u_hat = (g, 1, 0) / sqrt(g^2 + 1) with GELU written out independently;
    the loss 1 - (u_hat . u*)^2 is the same for u* and -u*."""
    K, H = 1, 1
    # W1, b1, W2, b2, W3 (3x1), b3
    P = np.array([1.0, 0.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0])
    gelu = lambda x: 0.5 * x * (1 + math.tanh(math.sqrt(2 / math.pi) * (x + 0.044715 * x ** 3)))
    for x in (-1.3, 0.0, 0.7, 2.5):
        g = gelu(gelu(x))
        u, _, _ = O.mlp(P, np.array([[x]]), H=H)
        assert np.allclose(u[0], np.array([g, 1.0, 0.0]) / math.hypot(g, 1.0), atol=1e-15)
    rng = np.random.default_rng(2)
    Pr = rng.normal(size=O.mlp_num_params(5, 4))
    X = rng.normal(size=(3, 5))
    U = rng.normal(size=(3, 3))
    _, L1, g1 = O.mlp(Pr, X, U, H=4, want_grad=True)
    _, L2, g2 = O.mlp(Pr, X, -U, H=4, want_grad=True)
    assert L1 == pytest.approx(L2, rel=1e-14)
    assert np.allclose(g1, g2, atol=1e-14)
