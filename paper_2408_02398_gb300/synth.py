"""Seeded synthetic inputs for tensorial template matching (TTM).

This module only *makes inputs*: random numbers, templates, noise volumes and
planted copies. It holds none of the matching method's arithmetic (no filter,
mask, normalisation, tensor field, correlation or maximisation), so the CPU
oracle and the CUDA path can both be fed from it without sharing code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
turned into uniforms on [0, 1) with 53 bits and into normals with the
Box-Muller transform. Every draw is addressed by (seed, stream, counter), so
the same inputs are produced on any machine.

Workload recipes follow the synthetic experiments of Sec. 5.1 (templates
planted at random rotations in a noisy tomogram): a template is a sum of six
anisotropic Gaussians, noise is white or Gaussian-low-passed, copies are
planted at uniformly random rotations with trilinear resampling.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# named sub-streams so that changing one draw never shifts another
STREAM_NOISE = 1
STREAM_TEMPLATE = 2
STREAM_PLACE = 3
STREAM_ROT = 4
STREAM_MISC = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix64(s)[0]


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0,1) from SplitMix64 counters offset+1 .. offset+n."""
    key = _stream_key(seed, stream)
    out = np.empty(n, dtype=np.float64)
    chunk = 1 << 24
    with np.errstate(over="ignore"):
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            ctr = np.arange(offset + s + 1, offset + e + 1, dtype=np.uint64)
            z = key + ctr * _GOLDEN
            out[s:e] = (_mix64(z) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return out


def normals(seed: int, stream: int, n: int, dtype=np.float64) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs."""
    out = np.empty(n, dtype=dtype)
    half = (n + 1) // 2
    chunk = 1 << 23
    for s in range(0, half, chunk):
        e = min(half, s + chunk)
        u = uniforms(seed, stream, 2 * (e - s), offset=2 * s)
        r = np.sqrt(-2.0 * np.log1p(-u[0::2]))
        th = 2.0 * math.pi * u[1::2]
        z0 = r * np.cos(th)
        z1 = r * np.sin(th)
        lo = 2 * s
        both = np.empty(2 * (e - s))
        both[0::2] = z0
        both[1::2] = z1
        m = min(n - lo, both.size)
        out[lo:lo + m] = both[:m]
    return out


def shoemake_quats(u: np.ndarray) -> np.ndarray:
    """Uniform random unit quaternions (w,x,y,z) from rows of 3 uniforms
    (Shoemake, "Uniform random rotations", Graphics Gems III, 1992)."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2.0 * math.pi * u[:, 1]
    t2 = 2.0 * math.pi * u[:, 2]
    q = np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)
    return q


def quat_matrix(q) -> np.ndarray:
    """Rotation matrix acting on column vectors (x, y, z) for q = (w,x,y,z)."""
    w, x, y, z = (float(v) for v in q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def resample_rotated(vol: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Sample vol at R^T p about its centre (N//2 per axis), trilinear, zero
    outside; i.e. the copy of vol rotated by R. Used only to plant copies."""
    nz, ny, nx = vol.shape
    cz, cy, cx = nz // 2, ny // 2, nx // 2
    pz, py, px = np.meshgrid(np.arange(nz) - cz, np.arange(ny) - cy, np.arange(nx) - cx,
                             indexing="ij")
    P = np.stack([px.ravel(), py.ravel(), pz.ravel()]).astype(np.float64)  # (x,y,z)
    src = R.T @ P
    sx, sy, sz = src[0] + cx, src[1] + cy, src[2] + cz
    x0 = np.floor(sx).astype(np.int64)
    y0 = np.floor(sy).astype(np.int64)
    z0 = np.floor(sz).astype(np.int64)
    fx, fy, fz = sx - x0, sy - y0, sz - z0
    out = np.zeros(P.shape[1])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                xi, yi, zi = x0 + dx, y0 + dy, z0 + dz
                wgt = (fx if dx else 1 - fx) * (fy if dy else 1 - fy) * (fz if dz else 1 - fz)
                ok = (xi >= 0) & (xi < nx) & (yi >= 0) & (yi < ny) & (zi >= 0) & (zi < nz)
                vals = np.zeros_like(out)
                vals[ok] = vol[zi[ok], yi[ok], xi[ok]]
                out += wgt * vals
    return out.reshape(nz, ny, nx)


def gaussian_blob_template(n: int, seed: int, n_blobs: int = 6, centre_radius: float = 5.0,
                           std_lo: float = 1.0, std_hi: float = 3.0, index: int = 0) -> np.ndarray:
    """Cubic n^3 template: sum of n_blobs anisotropic Gaussians with centres
    uniform in a ball of radius centre_radius, per-axis std U[std_lo,std_hi]
    and uniform random orientation; normalised to max 1."""
    base = index * 64 * n_blobs
    u = uniforms(seed, STREAM_TEMPLATE, 64 * n_blobs, offset=base).reshape(n_blobs, 64)
    c = n // 2
    g = np.arange(n) - c
    pz, py, px = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([px, py, pz], axis=-1).astype(np.float64)
    out = np.zeros((n, n, n))
    for b in range(n_blobs):
        # centre uniform in a ball: direction from normals, radius ~ U^(1/3)
        zc = np.array([math.sqrt(-2 * math.log1p(-u[b, 2 * i])) *
                       math.cos(2 * math.pi * u[b, 2 * i + 1]) for i in range(3)])
        zc /= max(np.linalg.norm(zc), 1e-300)
        ctr = zc * centre_radius * u[b, 6] ** (1.0 / 3.0)
        std = std_lo + (std_hi - std_lo) * u[b, 7:10]
        R = quat_matrix(shoemake_quats(u[b, 10:13])[0])
        d = (P - ctr) @ R  # coordinates in the blob frame
        out += np.exp(-0.5 * np.sum((d / std) ** 2, axis=-1))
    return out / out.max()


def _smooth_step(d: np.ndarray, width: float) -> np.ndarray:
    """1 inside (d <= 0), 0 outside, a raised-cosine edge of the given width."""
    t = np.clip(d / width + 0.5, 0.0, 1.0)
    return 0.5 * (1.0 + np.cos(math.pi * t))


def cylinder_template(n: int, radius: float = 3.0, half_length: float = 7.0, edge: float = 1.5) -> np.ndarray:
    """Cubic n^3 template: a solid cylinder along z through the centre with
    soft edges (the simple shape of the synthetic study); max 1."""
    c = n // 2
    g = np.arange(n) - c
    pz, py, px = np.meshgrid(g, g, g, indexing="ij")
    rho = np.sqrt(px ** 2 + py ** 2)
    out = _smooth_step(rho - radius, edge) * _smooth_step(np.abs(pz) - half_length, edge)
    return out / out.max()


def l_shape_template(n: int, thick: float = 2.0, long_arm: float = 8.0, short_arm: float = 5.0,
                     edge: float = 1.5) -> np.ndarray:
    """Cubic n^3 template: an L of two square bars of half-thickness thick,
    one along +x (length long_arm) and one along +y (length short_arm) from a
    common corner, shifted so that its centre of mass sits at the template
    centre. Unequal arms leave it without rotational symmetry. Max 1."""
    c = n // 2
    g = np.arange(n) - c
    pz, py, px = np.meshgrid(g, g, g, indexing="ij")

    def bar(a, lo, hi, b1, b2):
        return (_smooth_step(np.maximum(lo - a, a - hi), edge) * _smooth_step(np.abs(b1) - thick, edge)
                * _smooth_step(np.abs(b2) - thick, edge))

    def shape(dx, dy):
        x, y = px - dx, py - dy
        return np.maximum(bar(x, -thick, long_arm, y, pz), bar(y, -thick, short_arm, x, pz))

    out = shape(0.0, 0.0)
    m = out.sum()
    cx, cy = float((out * px).sum() / m), float((out * py).sum() / m)
    out = shape(-cx, -cy)
    return out / out.max()


def grid_tomogram(tmpl: np.ndarray, per_axis: int, spacing: int, margin: int, seed: int,
                  snr: float | None, mask_radius: float):
    """The synthetic study's tomogram: per_axis^3 copies of tmpl on a regular
    grid (spacing voxels apart, margin voxels from the faces), each at a
    Shoemake-uniform rotation, plus white noise at the given SNR (in-mask
    variance of the copy / noise variance; None = noise-free). Returns
    (float32 volume, Planted)."""
    n = tmpl.shape[0]
    edge = 2 * margin + (per_axis - 1) * spacing + n
    shape = (edge, edge, edge)
    c0 = margin + n // 2
    ax = c0 + spacing * np.arange(per_axis)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    centres = np.stack([zz.ravel(), yy.ravel(), xx.ravel()], axis=1)
    quats = shoemake_quats(uniforms(seed, STREAM_ROT, 3 * len(centres)))
    vol = np.zeros(shape)
    plant(vol, np.asarray(tmpl, dtype=np.float64), centres, quats, 1.0)
    if snr is not None:
        m = sphere_mask_values(n, mask_radius)
        sigma = math.sqrt(float(np.var(np.asarray(tmpl, dtype=np.float64)[m])) / float(snr))
        vol += sigma * normals(seed, STREAM_NOISE, vol.size).reshape(shape)
    return vol.astype(np.float32), Planted(centres, quats, 1.0)


def lowpass_gaussian_periodic(vol: np.ndarray, sigma: float = 1.0, radius: int = 4) -> np.ndarray:
    """Separable periodic Gaussian low-pass (truncated at radius), used to
    colour the synthetic noise."""
    k = np.exp(-0.5 * (np.arange(-radius, radius + 1) / sigma) ** 2)
    k /= k.sum()
    out = vol
    for ax in range(3):
        acc = np.zeros_like(out)
        for j, kj in enumerate(k):
            acc += kj * np.roll(out, j - radius, axis=ax)
        out = acc
    return out


def sphere_mask_values(n: int, r: float) -> np.ndarray:
    """Binary sphere used only to measure a template's in-mask variance for an
    SNR target (input scaling, not the method's mask)."""
    c = n // 2
    g = np.arange(n) - c
    pz, py, px = np.meshgrid(g, g, g, indexing="ij")
    return (px * px + py * py + pz * pz) <= r * r + 1e-9


@dataclass
class Planted:
    centres: np.ndarray          # (P, 3) integer (z, y, x)
    quats: np.ndarray            # (P, 4) (w, x, y, z)
    amplitude: float


@dataclass
class Workload:
    tomo: np.ndarray             # float32 [Z][Y][X]
    template: np.ndarray         # float32 [N][N][N]
    mask_radius: float
    order_n: int
    planted: Planted
    name: str = ""
    meta: dict = field(default_factory=dict)


def place_centres(shape, n_tmpl: int, count: int, min_dist: float, seed: int,
                  tries: int = 100000) -> np.ndarray:
    """Random sequential addition of integer centres at least n_tmpl//2 from
    every border and min_dist apart; stops after `tries` draws."""
    Z, Y, X = shape
    h = n_tmpl // 2
    lo = np.array([h, h, h])
    hi = np.array([Z - (n_tmpl - h), Y - (n_tmpl - h), X - (n_tmpl - h)])
    if np.any(hi < lo):
        return np.zeros((0, 3), dtype=np.int64)
    u = uniforms(seed, STREAM_PLACE, 3 * tries).reshape(tries, 3)
    cand = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    acc = []
    md2 = min_dist * min_dist
    for c in cand:
        if acc:
            d2 = np.sum((np.asarray(acc) - c) ** 2, axis=1)
            if np.min(d2) < md2:
                continue
        acc.append(c)
        if len(acc) == count:
            break
    return np.asarray(acc, dtype=np.int64).reshape(-1, 3)


def plant(vol: np.ndarray, tmpl: np.ndarray, centres: np.ndarray, quats: np.ndarray,
          amplitude: float) -> None:
    """Add amplitude * (template rotated by q) centred at each centre."""
    n = tmpl.shape[0]
    h = n // 2
    for c, q in zip(centres, quats):
        rot = resample_rotated(tmpl.astype(np.float64), quat_matrix(q))
        z, y, x = (int(v) for v in c)
        vol[z - h:z - h + n, y - h:y - h + n, x - h:x - h + n] += amplitude * rot


def make_workload(shape, n_tmpl: int, mask_radius: float, order_n: int, copies: int,
                  seed: int, amplitude: float | None = None, snr: float | None = None,
                  lowpass: bool = False, name: str = "", template_index: int = 0) -> Workload:
    """Noise tomogram (sigma=1, optionally low-passed and rescaled to unit std)
    with `copies` planted templates at uniform random rotations. Give either a
    fixed amplitude (template max = 1) or an SNR = in-mask variance of the
    scaled template / noise variance."""
    tmpl = gaussian_blob_template(n_tmpl, seed, index=template_index)
    vol, planted = make_tomogram(shape, tmpl, mask_radius, copies, seed, amplitude=amplitude, snr=snr,
                                 lowpass=lowpass)
    return Workload(tomo=vol, template=tmpl.astype(np.float32), mask_radius=mask_radius, order_n=order_n,
                    planted=planted, name=name)


def make_tomogram(shape, tmpl: np.ndarray, mask_radius: float, copies: int, seed: int,
                  amplitude: float | None = None, snr: float | None = None, lowpass: bool = False):
    """Noise tomogram with `copies` planted copies of a given template (see
    make_workload); returns (float32 volume, Planted)."""
    Z, Y, X = shape
    n_tmpl = tmpl.shape[0]
    noise = normals(seed, STREAM_NOISE, Z * Y * X).reshape(Z, Y, X)
    if lowpass:
        noise = lowpass_gaussian_periodic(noise)
        noise /= noise.std()
    if amplitude is None:
        m = sphere_mask_values(n_tmpl, mask_radius)
        amplitude = math.sqrt(float(snr) / float(np.var(np.asarray(tmpl, dtype=np.float64)[m])))
    centres = place_centres(shape, n_tmpl, copies, 2.0 * mask_radius, seed)
    quats = shoemake_quats(uniforms(seed, STREAM_ROT, 3 * len(centres)))
    vol = noise
    plant(vol, np.asarray(tmpl, dtype=np.float64), centres, quats, amplitude)
    return vol.astype(np.float32), Planted(centres, quats, amplitude)


# ---------------------------------------------------------------------------
# Named workloads. The tensor orders, sizes, copy counts and noise levels are
# the ones the benchmark suite is defined on; "r" is the mask radius.

def workload_small(seed: int = 20240802) -> Workload:
    """64^3 white noise, 16^3 template, r=7, order 2, 4 copies at amplitude 0.5."""
    return make_workload((64, 64, 64), 16, 7.0, 2, 4, seed, amplitude=0.5,
                         name="ttm_n2_64cube_t16")


def workload_order4(seed: int = 20240803, shape=(200, 512, 512), copies: int = 300) -> Workload:
    """512x512x200 low-passed noise, 40^3 template, r=16, order 4, 300 copies at SNR 0.1."""
    return make_workload(shape, 40, 16.0, 4, copies, seed, snr=0.1, lowpass=True,
                         name="ttm_n4_512x512x200_t40")


def workload_order6(seed: int = 20240804, shape=(256, 1024, 1024), copies: int = 2000) -> Workload:
    """1024x1024x256 white noise, 48^3 template, r=19, order 6, 2000 copies
    (as many as fit at 2r spacing) at SNR 0.05."""
    return make_workload(shape, 48, 19.0, 6, copies, seed, snr=0.05, name="ttm_n6_1024x1024x256_t48")


@dataclass
class BatchWorkload:
    tomos: list                  # float32 [Z][Y][X] arrays of uneven sizes
    templates: list              # float32 [N][N][N]
    mask_radius: float
    order_n: int
    copies: list                 # planted copies per tomogram
    name: str = ""


def workload_batched(seed: int = 20240805, n_tomos: int = 64, n_templates: int = 8, n_tmpl: int = 32,
                     mask_radius: float = 12.0, lo: int = 96, hi: int = 256) -> BatchWorkload:
    """n_tomos sub-tomograms, each axis uniform in [lo, hi], white noise with
    20-80 planted copies each (the template of each copy drawn uniformly
    from n_templates distinct n_tmpl^3 templates) at SNR 0.1; order 4."""
    templates = [gaussian_blob_template(n_tmpl, seed, index=j) for j in range(n_templates)]
    m = sphere_mask_values(n_tmpl, mask_radius)
    amps = [math.sqrt(0.1 / float(np.var(t[m]))) for t in templates]
    u = uniforms(seed, STREAM_MISC, 4 * n_tomos).reshape(n_tomos, 4)
    tomos, copies = [], []
    for i in range(n_tomos):
        shape = tuple(int(lo + math.floor(u[i, a] * (hi - lo + 1))) for a in range(3))
        count = int(20 + math.floor(u[i, 3] * 61))
        s = seed * 1000 + i + 1
        Z, Y, X = shape
        vol = normals(s, STREAM_NOISE, Z * Y * X).reshape(shape)
        centres = place_centres(shape, n_tmpl, count, 2.0 * mask_radius, s)
        quats = shoemake_quats(uniforms(s, STREAM_ROT, 3 * len(centres)))
        which = np.floor(uniforms(s, STREAM_PLACE, len(centres), offset=10 ** 6) * n_templates).astype(int)
        for j in range(n_templates):
            sel = which == j
            if np.any(sel):
                plant(vol, templates[j], centres[sel], quats[sel], amps[j])
        tomos.append(vol.astype(np.float32))
        copies.append(len(centres))
    return BatchWorkload(tomos=tomos, templates=[t.astype(np.float32) for t in templates],
                         mask_radius=mask_radius, order_n=4, copies=copies,
                         name="ttm_n4_batched_%dx[%d-%d]^3_%dtmpl_t%d" % (n_tomos, lo, hi, n_templates, n_tmpl))


def random_tensors(seed: int, count: int, K: int) -> np.ndarray:
    """count x K standard-normal tensor components (maximiser tests)."""
    return normals(seed, STREAM_MISC, count * K).reshape(count, K)
