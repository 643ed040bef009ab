"""FP64 CPU oracle for tensorial template matching -- TEST INFRASTRUCTURE.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package. It wraps ``ttm_oracle.c`` (plain C, double
precision, direct spatial sums, no FFT) through ctypes; the shared object is
compiled with gcc on first use (or by ``oracle.build.build()``). It shares no
code with the CUDA library.

Every function takes and returns numpy arrays; see ``ttm_oracle.c`` for the
equation each step follows.
"""
from __future__ import annotations

import ctypes as C
import os

import math

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


_d = C.c_double
_i = C.c_int
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int)
_pi64 = C.POINTER(C.c_int64)
_pi32 = C.POINTER(C.c_int32)


def _declare(L):
    sig = {
        "oracle_num_threads": (_i, []),
        "oracle_set_threads": (None, [_i]),
        "oracle_num_components": (_i, [_i, _i]),
        "oracle_multi_indices": (_i, [_i, _i, _pi]),
        "oracle_multiplicities": (None, [_i, _i, _pd]),
        "oracle_filter3": (None, [_pd, _i, _i, _i, _d, _pd]),
        "oracle_mask": (_d, [_i, _i, _i, _d, _d, _pd]),
        "oracle_normalise_template": (_d, [_pd, _i, _i, _i, _pd, _d, _pd]),
        "oracle_superfib_psi": (_d, []),
        "oracle_superfib": (None, [_i64, _pd]),
        "oracle_quat_mul": (None, [_pd, _pd, _pd]),
        "oracle_quat_to_rot": (None, [_pd, _pd]),
        "oracle_cube_rotations": (None, [_pd]),
        "oracle_symmetrise_cube": (None, [_pd, _i64, _pd]),
        "oracle_rotate_template": (None, [_pd, _i, _i, _i, _pd, _pd]),
        "oracle_tensor_field": (_i, [_pd, _i, _i, _i, _pd, _i64, _i, _i, _pd]),
        "oracle_global_variance": (_d, [_pd, _i64]),
        "oracle_mean_square": (_d, [_pd, _i64]),
        "oracle_local_w": (None, [_pd, _i, _i, _i, _pd, _i, _i, _i, _i, _d, _pi64, _i64, _pd,
                                  _pd, _pd]),
        "oracle_correlate": (None, [_pd, _i, _i, _i, _pd, _i, _i, _i, _i, _i, _pi64, _i64, _pd,
                                    _pd]),
        "oracle_frobenius": (None, [_pd, _i, _i, _i, _i64, _pd]),
        "oracle_sample_directions": (None, [_i, _i, _pd]),
        "oracle_maximise": (None, [_pd, _i64, _i, _i, _i, _pd, _pd, _pd, _pd]),
        "oracle_poly_eval": (_d, [_pd, _i, _i, _pd, _pd, _pd]),
        "oracle_find_peaks": (_i, [_pd, _i, _i, _i, _i, _i, _i, _i, _i, _i, _i, _d, _pi64, _pd]),
        "oracle_tm": (None, [_pd, _i, _i, _i, _pd, _i, _i, _i, _pd, _i64, _i, _pi64, _i64, _pd,
                             _pd, _pi32]),
        "oracle_mlp_num_params": (_i64, [_i, _i]),
        "oracle_mlp": (_d, [_pd, _i, _i, _pd, _pd, _i64, _pd, _pd]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=_pd):
    if a is None:
        return None
    return a.ctypes.data_as(t)


# ---------------------------------------------------------------- basics ---

def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def num_components(n: int, d: int = 3) -> int:
    return lib().oracle_num_components(n, d)


def multi_indices(n: int, d: int = 3) -> np.ndarray:
    K = num_components(n, d)
    a = np.zeros((K, d), dtype=np.int32)
    lib().oracle_multi_indices(n, d, a.ctypes.data_as(_pi))
    return a


def multiplicities(n: int, d: int = 3) -> np.ndarray:
    K = num_components(n, d)
    m = np.zeros(K)
    lib().oracle_multiplicities(n, d, _p(m))
    return m


def filter3(f, a: float = 0.2) -> np.ndarray:
    f = _f64(f)
    g = np.empty_like(f)
    Z, Y, X = f.shape
    lib().oracle_filter3(_p(f), Z, Y, X, a, _p(g))
    return g


def mask(shape, r: float, soft: float = 0.0):
    tz, ty, tx = shape
    m = np.zeros(shape)
    M = lib().oracle_mask(tz, ty, tx, r, soft, _p(m))
    return m, M


def normalise_template(t, m, a: float = 0.2):
    t = _f64(t)
    m = _f64(m)
    tp = np.empty_like(t)
    tz, ty, tx = t.shape
    den = lib().oracle_normalise_template(_p(t), tz, ty, tx, _p(m), a, _p(tp))
    return tp, den


# -------------------------------------------------------------- rotations --

def superfib_psi() -> float:
    return lib().oracle_superfib_psi()


def superfib(N: int) -> np.ndarray:
    q = np.zeros((N, 4))
    lib().oracle_superfib(N, _p(q))
    return q


def quat_mul(p, q) -> np.ndarray:
    p, q = _f64(p), _f64(q)
    o = np.zeros(4)
    lib().oracle_quat_mul(_p(p), _p(q), _p(o))
    return o


def quat_to_rot(q) -> np.ndarray:
    q = _f64(q)
    R = np.zeros(9)
    lib().oracle_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def cube_rotations() -> np.ndarray:
    q = np.zeros((24, 4))
    lib().oracle_cube_rotations(_p(q))
    return q


def symmetrise_cube(base) -> np.ndarray:
    base = _f64(base).reshape(-1, 4)
    out = np.zeros((base.shape[0] * 24, 4))
    lib().oracle_symmetrise_cube(_p(base), base.shape[0], _p(out))
    return out


def rotation_set(n_base: int = 2048, cube: bool = True) -> np.ndarray:
    """Default quadrature for Eq. 9: super-Fibonacci samples, optionally
    symmetrised by the cube group (24 * n_base rotations)."""
    b = superfib(n_base)
    return symmetrise_cube(b) if cube else b


def rotate_template(t, q) -> np.ndarray:
    t = _f64(t)
    q = _f64(q)
    o = np.empty_like(t)
    tz, ty, tx = t.shape
    lib().oracle_rotate_template(_p(t), tz, ty, tx, _p(q), _p(o))
    return o


# ---------------------------------------------------------------- method ---

def tensor_field(tp, quats, n: int, d: int = 3) -> np.ndarray:
    tp = _f64(tp)
    quats = _f64(quats).reshape(-1, 4)
    tz, ty, tx = tp.shape
    K = num_components(n, d)
    T = np.zeros((K, tz, ty, tx))
    lib().oracle_tensor_field(_p(tp), tz, ty, tx, _p(quats), quats.shape[0], n, d, _p(T))
    return T


def global_variance(g) -> float:
    g = _f64(g)
    return lib().oracle_global_variance(_p(g), g.size)


def mean_square(g) -> float:
    g = _f64(g)
    return lib().oracle_mean_square(_p(g), g.size)


def var_floor(g, M: float) -> float:
    """Local variances at or below this give w = 0: 1e-8 * M * mean(g^2), the
    level of an (almost) empty window relative to the volume's energy, where
    the LNCC of an FP32 correlation is not resolved."""
    return 1e-8 * M * mean_square(g)


def _vox(vox, shape):
    if vox is None:
        return np.arange(int(np.prod(shape)), dtype=np.int64)
    return np.ascontiguousarray(vox, dtype=np.int64).ravel()


def valid_voxels(shape, tshape) -> np.ndarray:
    """Linear indices of the valid interior: voxels whose whole template
    window lies inside the volume."""
    Z, Y, X = shape
    tz, ty, tx = tshape
    z = np.arange(tz // 2, Z - (tz - tz // 2) + 1)
    y = np.arange(ty // 2, Y - (ty - ty // 2) + 1)
    x = np.arange(tx // 2, X - (tx - tx // 2) + 1)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return ((zz * Y + yy) * X + xx).ravel().astype(np.int64)


def local_w(g, m, vox=None, periodic: bool = False, floor: float | None = None):
    """w, S1, S2 of Eq. 2 at the voxels vox (linear indices)."""
    g = _f64(g)
    m = _f64(m)
    v = _vox(vox, g.shape)
    if floor is None:
        floor = var_floor(g, float(m.sum()))
    w = np.zeros(v.size)
    S1 = np.zeros(v.size)
    S2 = np.zeros(v.size)
    Z, Y, X = g.shape
    tz, ty, tx = m.shape
    lib().oracle_local_w(_p(g), Z, Y, X, _p(m), tz, ty, tx, int(periodic), floor,
                         _p(v, _pi64), v.size, _p(w), _p(S1), _p(S2))
    return w, S1, S2


def correlate(g, T, vox=None, periodic: bool = False, w=None) -> np.ndarray:
    """[K][nvox] correlation (Eq. 5) of g with each component of T, times w."""
    g = _f64(g)
    T = _f64(T)
    if T.ndim == 3:
        T = T[None]
    v = _vox(vox, g.shape)
    K, tz, ty, tx = T.shape
    Z, Y, X = g.shape
    out = np.zeros((K, v.size))
    wv = None if w is None else _f64(w)
    lib().oracle_correlate(_p(g), Z, Y, X, _p(T), K, tz, ty, tx, int(periodic), _p(v, _pi64),
                           v.size, _p(wv), _p(out))
    return out


def frobenius(C, n: int, d: int = 3) -> np.ndarray:
    C = _f64(C)
    K, nv = C.shape
    F = np.zeros(nv)
    lib().oracle_frobenius(_p(C), K, n, d, nv, _p(F))
    return F


def sample_directions(d: int, ns: int) -> np.ndarray:
    U = np.zeros((ns, d))
    lib().oracle_sample_directions(d, ns, _p(U))
    return U


def maximise(C, n: int, d: int = 3, nsamples: int = 20000, with_curvature: bool = False):
    """Per voxel (columns of C = [K][nvox]): score max_u C.u^n, canonical
    argmax u (nvox x d) and the best distinct second local maximum; with
    with_curvature also the curvature at the maximum (smallest eigenvalue of
    minus the Riemannian Hessian)."""
    C = _f64(C)
    K, nv = C.shape
    s = np.zeros(nv)
    u = np.zeros((nv, d))
    sec = np.zeros(nv)
    curv = np.zeros(nv) if with_curvature else None
    lib().oracle_maximise(_p(C), nv, n, d, nsamples, _p(s), _p(u), _p(sec), _p(curv))
    if with_curvature:
        return s, u, sec, curv
    return s, u, sec


def poly_eval(c, n: int, d: int, u):
    c = _f64(c)
    u = _f64(u)
    g = np.zeros(d)
    H = np.zeros(d * d)
    p = lib().oracle_poly_eval(_p(c), n, d, _p(u), _p(g), _p(H))
    return p, g, H.reshape(d, d)


def find_peaks(s, box, P: int, min_dist: float):
    """box = (z0, z1, y0, y1, x0, x1); returns (linear indices, values)."""
    s = _f64(s)
    Z, Y, X = s.shape
    idx = np.zeros(P, dtype=np.int64)
    val = np.zeros(P)
    got = lib().oracle_find_peaks(_p(s), Z, Y, X, *[int(b) for b in box], P, float(min_dist),
                                  _p(idx, _pi64), _p(val))
    return idx[:got], val[:got]


def tm(g, tp, quats, vox=None, periodic: bool = False, w=None):
    """Classical TM (Eqs. 1, 6, 7): best LNCC and first arg-max rotation index."""
    g = _f64(g)
    tp = _f64(tp)
    quats = _f64(quats).reshape(-1, 4)
    v = _vox(vox, g.shape)
    Z, Y, X = g.shape
    tz, ty, tx = tp.shape
    best = np.zeros(v.size)
    bidx = np.zeros(v.size, dtype=np.int32)
    wv = None if w is None else _f64(w)
    lib().oracle_tm(_p(g), Z, Y, X, _p(tp), tz, ty, tx, _p(quats), quats.shape[0],
                    int(periodic), _p(v, _pi64), v.size, _p(wv), _p(best), _p(bidx, _pi32))
    return best, bidx


def ball_offsets(r_s: float) -> np.ndarray:
    """Alg. 3's candidates around a peak in the order they are visited: the
    peak itself, then every other offset d with |d| <= r_s in (z, y, x)
    lexicographic order; rows (dz, dy, dx)."""
    R = int(math.floor(r_s))
    out = [(0, 0, 0)]
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                if (dz, dy, dx) != (0, 0, 0) and dz * dz + dy * dy + dx * dx <= r_s * r_s:
                    out.append((dz, dy, dx))
    return np.array(out, dtype=np.int64)


def ttm_refine(pr, field, n: int, peaks, r_s: float = 3.0, nsamples: int = 20000):
    """TTM-ref (Sec. 3.3, Alg. 3) with d' = 4: for each peak, every ball
    voxel inside the valid interior gets its optimal rotation from its own C
    (Eq. 8, then the maximiser over unit quaternions) and the LNCC at that
    single rotation (Eq. 1 / Eq. 7 via tm); the first strictly highest
    voxel in the order of ball_offsets is kept. pr is a Prepared set, field
    the d' = 4 tensor field. Returns (indices, quaternions [P][4], LNCC [P],
    per-peak lists of (candidate indices, their LNCC))."""
    Z, Y, X = pr.g.shape
    tz, ty, tx = pr.tshape
    lo = np.array([tz // 2, ty // 2, tx // 2])
    hi = np.array([Z - (tz - tz // 2), Y - (ty - ty // 2), X - (tx - tx // 2)])
    offs = ball_offsets(r_s)
    idx, quats, vals, cands = [], [], [], []
    for pk in np.asarray(peaks, dtype=np.int64):
        c0 = np.array([pk // (Y * X), (pk // X) % Y, pk % X])
        pos = c0[None, :] + offs
        ok = np.all((pos >= lo) & (pos <= hi), axis=1)
        if not ok[0]:
            raise ValueError("peak outside the valid interior")
        pos = pos[ok]
        vox = (pos[:, 0] * Y + pos[:, 1]) * X + pos[:, 2]
        w, _, _ = local_w(pr.g, pr.m, vox, False, pr.floor)
        C = correlate(pr.g, field, vox, False, w)
        _, q, _ = maximise(C, n, 4, nsamples)
        c = np.array([tm(pr.g, pr.tp, q[k], vox[k:k + 1], False, w[k:k + 1])[0][0] for k in range(vox.size)])
        best = 0
        for k in range(1, vox.size):
            if c[k] > c[best]:
                best = k
        idx.append(int(vox[best]))
        quats.append(q[best])
        vals.append(float(c[best]))
        cands.append((vox, c))
    return np.array(idx, dtype=np.int64), np.array(quats).reshape(-1, 4), np.array(vals), cands


# ------------------------------------------------------- learned start ---

def mlp_num_params(K: int, H: int = 128) -> int:
    return int(lib().oracle_mlp_num_params(K, H))


def mlp(params, X, U=None, H: int = 128, want_grad: bool = False):
    """MLP K -> H -> H -> 3 (GELU), normalised output: returns (u_hat [n][3],
    summed loss 1 - (u_hat . u*)^2 or None, summed gradient or None)."""
    params = _f64(params)
    X = _f64(X)
    n, K = X.shape
    Ud = None if U is None else _f64(U)
    out = np.zeros((n, 3))
    grad = np.zeros(params.size) if want_grad else None
    loss = lib().oracle_mlp(_p(params), K, H, _p(X), _p(Ud), n, _p(out), _p(grad))
    return out, (loss if U is not None else None), grad


# ------------------------------------------------------------ pipelines ---

class Prepared:
    """Filtered tomogram, mask and normalised template of one (tomogram,
    template, mask radius, filter) set, in FP64."""

    def __init__(self, tomo, tmpl, r: float, a: float = 0.2, soft: float = 0.0):
        self.g = filter3(tomo, a)
        self.m, self.M = mask(tmpl.shape, r, soft)
        self.tp, self.sigma_t = normalise_template(tmpl, self.m, a)
        self.floor = var_floor(self.g, self.M)
        self.tshape = tuple(tmpl.shape)


def ttm(tomo, tmpl, r: float, n: int, quats, vox=None, periodic: bool = False, d: int = 3,
        a: float = 0.2, nsamples: int = 20000, field=None, maximise_too: bool = True):
    """The whole path at the voxels vox: C (Eq. 8), Frobenius map, score and
    orientation. Returns a dict."""
    pr = Prepared(tomo, tmpl, r, a)
    T = tensor_field(pr.tp, quats, n, d) if field is None else field
    v = valid_voxels(pr.g.shape, pr.tshape) if vox is None else _vox(vox, pr.g.shape)
    w, S1, S2 = local_w(pr.g, pr.m, v, periodic, pr.floor)
    C = correlate(pr.g, T, v, periodic, w)
    out = {"vox": v, "w": w, "S1": S1, "S2": S2, "C": C, "T": T, "F": frobenius(C, n, d),
           "prepared": pr}
    if maximise_too:
        s, u, sec, curv = maximise(C, n, d, nsamples, with_curvature=True)
        out.update(score=s, orient=u, second=sec, curv=curv)
    return out


if os.environ.get("TTM_ORACLE_THREADS"):
    set_threads(int(os.environ["TTM_ORACLE_THREADS"]))
