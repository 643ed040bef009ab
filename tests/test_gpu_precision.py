"""Mixed-precision correlate: template spectra and the K-component work
buffer stored as FP16 or BF16 pairs with per-component scaling, FP32
arithmetic, FP64 local variance. Errors against the FP64 oracle are bounded
from the storage format: three roundings (stored spectrum, z-pass and y-pass
stores) of unit roundoff u each, u = 2^-11 (FP16) or 2^-8 (BF16), so C is
held to a relative L2 error of 3u and a max error of 3u max|C|. The score
max_u C . u^n is 1-Lipschitz in the Frobenius norm, so at every voxel its
error is held to ||C_gpu(x) - C_ref(x)||_F plus the maximiser's own
tolerance (1e-4, the FP32 form's: where two local maxima lie closer than
that, either may be returned)."""
import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

UNIT = {1: 2.0 ** -11, 2: 2.0 ** -8}   # TTM_PREC_FP16_SPECTRA, TTM_PREC_BF16_SPECTRA


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


CASES = [
    ((24, 20, 28), 7, 3.0, 2),       # Stockham lengths on every axis
    ((32, 30, 36), 9, 4.0, 6),
    ((128, 128, 256), 11, 5.0, 6),   # register lengths
    ((64, 128, 128), 24, 9.0, 6),
]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape,N,r,n", CASES)
def test_mixed_precision_vs_oracle(T, ctx, shape, N, r, n, prec):
    V = int(np.prod(shape))
    tomo = synth.normals(11 + N, 1, V).reshape(shape).astype(np.float32)
    tmpl = synth.gaussian_blob_template(N, seed=N + 1)
    field = oracle_field(tmpl, r, n, 16)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=16)
    vox = np.sort(np.random.default_rng(N).choice(V, size=min(V, 800), replace=False))
    pr = O.Prepared(tomo.astype(np.float64), tmpl, r)
    w, _, _ = O.local_w(pr.g, pr.m, vox, periodic=True, floor=pr.floor)
    Cref = O.correlate(pr.g, field, vox, periodic=True, w=w)
    sref, _, _ = O.maximise(Cref, n, 3, nsamples=20000)
    K = field.shape[0]
    plan = T.Plan(ctx, dev(field, torch.float64), p, shape, precision=prec)
    d_C = torch.empty((K,) + shape, device="cuda")
    T.ttm_correlate(plan, dev(tomo), d_C)
    d_s = torch.empty(shape, device="cuda")
    d_u = torch.empty((3,) + shape, device="cuda")
    T.ttm_peak_map(plan, d_C, d_s, d_u)
    got = d_C.cpu().numpy().reshape(K, -1)[:, vox]
    u = UNIT[prec]
    assert np.linalg.norm(got - Cref) <= 3 * u * np.linalg.norm(Cref)
    assert np.abs(got - Cref).max() <= 3 * u * np.abs(Cref).max()
    s = d_s.cpu().numpy().ravel()[vox]
    dF = O.frobenius(got.astype(np.float64) - Cref, n)
    assert np.all(np.abs(s - sref) <= dF + 1e-4)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_planted_peaks(T, ctx, prec):
    """On the 64^3 order-2 workload the reduced-precision score map gives the
    same top peaks, bit for bit, as the FP32 one."""
    wl = synth.workload_small()
    p = T.params(order_n=2, mask_radius=wl.mask_radius, n_rot_base=256)
    K = T.ttm_num_components(2)
    tm = dev(wl.template)
    d_field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, tm, p, d_field)
    out = {}
    for pr in (0, prec):
        plan = T.Plan(ctx, d_field, p, wl.tomo.shape, precision=pr)
        d_C = torch.empty((K,) + wl.tomo.shape, device="cuda")
        T.ttm_correlate(plan, dev(wl.tomo), d_C)
        d_s = torch.empty(wl.tomo.shape, device="cuda")
        d_u = torch.empty((3,) + wl.tomo.shape, device="cuda")
        T.ttm_peak_map(plan, d_C, d_s, d_u)
        out[pr] = T.ttm_find_peaks(plan, d_s, 4, 2 * wl.mask_radius)
    assert np.array_equal(out[0][0], out[prec][0])
    assert np.allclose(out[0][1], out[prec][1], atol=3 * UNIT[prec])


def test_unknown_precision_rejected(T, ctx):
    field = torch.zeros((6, 5, 5, 5), dtype=torch.float64, device="cuda")
    p = T.params(order_n=2, mask_radius=2.0, n_rot_base=4)
    with pytest.raises(T.TTMError):
        T.Plan(ctx, field, p, (16, 16, 16), precision=7)
