"""The allocation-free Find Peaks entry point against ttm_find_peaks.

Both are called through the C ABI on the same device maps; peak lists are
index work and must agree exactly, on two calls in a row (the second call
reuses the library's fixed scratch array that the first one filled)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


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


def plan_for(T, ctx, shape, t=5, n=2):
    """A plan whose only use here is its valid box and candidate buffer."""
    K = T.ttm_num_components(n, 3)
    field = torch.zeros((K, t, t, t), dtype=torch.float64, device="cuda")
    p = T.params(order_n=n, mask_radius=2.0, n_rot_base=4)
    return T.Plan(ctx, field, p, shape)


def smooth_map(shape, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(shape)
    for ax in range(3):   # a few box blurs: peaks a few voxels apart
        s = (np.roll(s, 1, ax) + s + np.roll(s, -1, ax)) / 3.0
    s = s.astype(np.float32)
    s[6:9, 6:9, 6:9] = s.max() + 1.0     # a plateau: one peak at its lowest index
    s[20, 20, 20] = s[24, 24, 24] = s.max() + 0.5   # two equal values
    return s


@pytest.mark.parametrize("P,md", [(10, 4.0), (200, 2.5), (1000, 0.0), (0, 1.0), (5000, 6.0)])
def test_noalloc_matches_find_peaks_two_calls(T, ctx, P, md):
    shape = (40, 48, 56)
    plan = plan_for(T, ctx, shape)
    box = plan.valid_box()
    d = torch.as_tensor(smooth_map(shape, 11), device="cuda")
    ri, rv = T.ttm_find_peaks(plan, d, P, md)
    for _ in range(2):
        gi, gv = T.ttm_find_peaks_noalloc(ctx, d, box, P, md)
        assert np.array_equal(gi, ri)
        assert np.array_equal(gv, rv)
    if P:
        assert len(ri) > 0


def test_noalloc_white_noise_many_candidates(T, ctx):
    """White noise: tens of thousands of candidates, ties broken by index."""
    shape = (64, 96, 80)
    plan = plan_for(T, ctx, shape)
    box = plan.valid_box()
    s = np.random.default_rng(3).integers(0, 50, size=shape).astype(np.float32)   # many ties
    d = torch.as_tensor(s, device="cuda")
    ri, rv = T.ttm_find_peaks(plan, d, 3000, 3.0)
    for _ in range(2):
        gi, gv = T.ttm_find_peaks_noalloc(ctx, d, box, 3000, 3.0)
        assert np.array_equal(gi, ri) and np.array_equal(gv, rv)


def test_noalloc_rejects_sizes_beyond_capacity(T, ctx):
    d = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(T.TTMError) as e:
        T.ttm_find_peaks_noalloc(ctx, d, (0, 8, 0, 8, 0, 8), 16385, 1.0)
    assert e.value.code == 2   # TTM_E_SHAPE
    assert "16384" in str(e.value)
    # 68^3 isolated maxima (every voxel with three even coordinates) > 262144
    s = torch.zeros((136, 136, 136), dtype=torch.float32, device="cuda")
    s[::2, ::2, ::2] = 1.0
    with pytest.raises(T.TTMError) as e:
        T.ttm_find_peaks_noalloc(ctx, s, (0, 136, 0, 136, 0, 136), 10, 1.0)
    assert e.value.code == 2 and "262144" in str(e.value)
    # a smaller box of the same map fits: 32^3 candidates, all value 1,
    # so the lowest indices win, min_dist 3 keeps every other one per axis
    gi, gv = T.ttm_find_peaks_noalloc(ctx, s, (0, 64, 0, 64, 0, 64), 100, 3.0)
    assert len(gi) == 100 and np.all(gv == 1.0)
    assert gi[0] == 0
    z, y, x = np.unravel_index(gi, (136, 136, 136))
    assert np.all(z % 2 == 0) and np.all(y % 2 == 0) and np.all(x % 2 == 0)


def test_noalloc_bad_box(T, ctx):
    d = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(T.TTMError):
        T.ttm_find_peaks_noalloc(ctx, d, (0, 9, 0, 8, 0, 8), 4, 1.0)
    gi, _ = T.ttm_find_peaks_noalloc(ctx, d, (3, 3, 0, 8, 0, 8), 4, 1.0)   # empty box
    assert len(gi) == 0
