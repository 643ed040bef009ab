"""Block processing with halos and Merge Peaks (Sec. 3.4) on the GPU: the
peak list of a tomogram processed in z-slabs equals Find Peaks on the whole
tomogram (same candidates, same order; values up to the rounding of the
different FFT lengths), and its values equal the oracle's score at those
voxels."""
import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("slab_z,map_kind,dprime", [(9, 0, 3), (23, 1, 3), (200, 0, 3), (7, 0, 4)])
def test_blocked_peaks_equal_whole_volume(T, ctx, slab_z, map_kind, dprime):
    shape = (70, 48, 56)
    N, r, n = 12, 5.0, 4
    tmpl = synth.gaussian_blob_template(N, seed=41).astype(np.float32)
    vol, pl = synth.make_tomogram(shape, tmpl, r, 6, seed=42, amplitude=1.0)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=32, dprime=dprime)
    K = T.ttm_num_components(n, dprime)
    field = torch.empty((K, N, N, N), dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, field)
    plan = T.Plan(ctx, field, p, shape)
    C = torch.empty((K,) + shape, device="cuda")
    T.ttm_correlate(plan, dev(vol), C)
    s = torch.empty(shape, device="cuda")
    u = torch.empty((dprime,) + shape, device="cuda")
    F = torch.empty(shape, device="cuda")
    T.ttm_peak_map(plan, C, s, u, F)
    torch.cuda.synchronize()
    P, md = 40, 2 * r
    wi, wv = T.ttm_find_peaks(plan, s if map_kind == 0 else F, P, md)
    bi, bv = T.ttm_blocked_peaks(ctx, field, p, vol, slab_z, P, md, map_kind=map_kind)
    assert len(bi) == len(wi) > 10
    assert np.abs(bv - wv).max() <= 1e-5 * max(1.0, np.abs(wv).max())
    assert list(bi) == list(wi)
    if map_kind == 0 and dprime == 3:
        # the planted copies are found (within the few-voxel shift of the score
        # peaks that Sec. 3.3 describes and TTM-ref corrects), and the values
        # are the oracle's scores there
        pz = np.stack(np.unravel_index(bi[:12], shape), axis=1)
        near = [np.min(np.linalg.norm(pz - np.asarray(c), axis=1)) <= 4.0 for c in pl.centres]
        assert sum(near) >= 4
        res = O.ttm(vol.astype(np.float64), tmpl.astype(np.float64), r, n, O.rotation_set(32), vox=bi[:10],
                    nsamples=20000)
        assert np.abs(bv[:10] - res["score"]).max() <= S_TOL


def test_blocked_peaks_rejects_bad_arguments(T, ctx):
    tmpl = synth.gaussian_blob_template(8, seed=1).astype(np.float32)
    p = T.params(order_n=2, mask_radius=3.0, n_rot_base=8)
    field = torch.empty((6, 8, 8, 8), dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, field)
    vol = np.zeros((20, 20, 20), dtype=np.float32)
    with pytest.raises(T.TTMError):
        T.ttm_blocked_peaks(ctx, field, p, vol, 0, 5, 4.0)
    with pytest.raises(T.TTMError):
        T.ttm_blocked_peaks(ctx, field, p, vol[:5], 4, 5, 4.0)


def test_blocked_session_reused_and_equal_to_one_shot(T, ctx):
    """A block-processing session kept across tomograms (plans, buffers and
    the copy stream made once): two different tomograms run through one
    session give the one-shot call's lists, also from pinned host memory."""
    shape = (70, 48, 56)
    N, r, n = 12, 5.0, 4
    tmpl = synth.gaussian_blob_template(N, seed=43).astype(np.float32)
    p = T.params(order_n=n, mask_radius=r, n_rot_base=32)
    K = T.ttm_num_components(n)
    field = torch.empty((K, N, N, N), dtype=torch.float64, device="cuda")
    T.ttm_build_tensor_field(ctx, dev(tmpl), p, field)
    sess = T.Blocked(ctx, field, p, shape, 24)
    for seed in (44, 45):
        vol, _ = synth.make_tomogram(shape, tmpl, r, 6, seed=seed, amplitude=1.0)
        oi, ov = T.ttm_blocked_peaks(ctx, field, p, vol, 24, 30, 2 * r)
        si, sv = sess.run(vol, 30, 2 * r)
        pi, pv = sess.run(torch.as_tensor(vol).pin_memory(), 30, 2 * r)
        assert list(si) == list(oi) and list(pi) == list(oi) and len(oi) > 10
        assert np.array_equal(sv, ov) and np.array_equal(pv, ov)
    with pytest.raises(ValueError):
        sess.run(np.zeros((10, 10, 10), np.float32), 5, 1.0)
