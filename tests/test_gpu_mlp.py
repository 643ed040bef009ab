"""Learned warm start on the GPU: the MLP's FP32 forward and gradient and its
BF16 tensor-core inference against the FP64 oracle, training on pairs that
the plain maximiser labels, and the learned maximiser against both the plain
maximiser (the reference for its error) and the oracle, including what it gains."""
import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

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


def unit_rows(rng, n, d):
    x = rng.standard_normal((n, d))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


@pytest.fixture(scope="module")
def net_and_data(T, ctx):
    """An MLP with perturbed (non-zero bias) parameters and random unit rows."""
    K = 28
    m = T.Mlp(ctx, K, seed=1)
    rng = np.random.default_rng(0)
    p = m.get_params().astype(np.float64) + 0.05 * rng.standard_normal(m.num_params)
    m.set_params(p.astype(np.float32))
    X = unit_rows(rng, 3000, K)
    U = unit_rows(rng, 3000, 3)
    return m, m.get_params().astype(np.float64), X, U


def test_mlp_forward_matches_oracle(T, net_and_data):
    m, p, X, U = net_and_data
    uo, _, _ = O.mlp(p, X.astype(np.float64))
    dU = torch.empty((len(X), 3), device="cuda")
    m.forward(dev(X), dU)
    assert np.abs(dU.cpu().numpy() - uo).max() <= 2e-5


def test_mlp_gradient_matches_oracle(T, net_and_data):
    """GPU backward (FP32, hand-written kernels) vs the oracle's FP64 one on
    identical weights and data."""
    m, p, X, U = net_and_data
    _, Lo, go = O.mlp(p, X.astype(np.float64), U.astype(np.float64), want_grad=True)
    g = torch.zeros(m.num_params, device="cuda")
    L = m.loss_grad(dev(X), dev(U), g)
    assert abs(L - Lo) <= 1e-6 * Lo
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-4 * np.abs(go).max()


def test_mlp_bf16_training_gradient_close_to_oracle(T, ctx, net_and_data):
    """TTM_MLP_BF16: the forward and backward products take BF16 operands on
    the tensor cores (FP32 accumulation). Loss and gradient against the
    oracle's FP64 ones on identical weights, within what BF16 rounding of
    the operands (unit roundoff 2^-8, three layers) allows; the gradient
    direction is kept (cosine > 0.999)."""
    m0, p, X, U = net_and_data
    m = T.Mlp(ctx, m0.K, seed=1)
    m.set_params(m0.get_params())
    m.set_precision(T.TTM_MLP_BF16)
    _, Lo, go = O.mlp(p, X.astype(np.float64), U.astype(np.float64), want_grad=True)
    g = torch.zeros(m.num_params, device="cuda")
    L = m.loss_grad(dev(X), dev(U), g)
    gb = g.cpu().numpy().astype(np.float64)
    assert abs(L - Lo) <= 1e-2 * Lo
    assert np.abs(gb - go).max() <= 5e-2 * np.abs(go).max()
    assert gb @ go / (np.linalg.norm(gb) * np.linalg.norm(go)) > 0.999
    m.set_precision(T.TTM_MLP_FP32)
    L32 = m.loss_grad(dev(X), dev(U), g)
    assert abs(L32 - Lo) <= 1e-6 * Lo
    with pytest.raises(T.TTMError):
        m.set_precision(2)


def test_mlp_bf16_inference_close_to_oracle(T, net_and_data):
    """Tensor-core inference (BF16 operands, FP32 accumulation, tanh.approx
    GELU): direction within a BF16 tolerance of the FP64 forward."""
    m, p, X, U = net_and_data
    uo, _, _ = O.mlp(p, X.astype(np.float64))
    dU = torch.empty((len(X), 3), device="cuda")
    m.infer(dev(X), dU)
    ub = dU.cpu().numpy()
    ang = np.degrees(np.arccos(np.clip(np.abs(np.sum(ub * uo, 1)), 0, 1)))
    assert ang.mean() <= 0.5 and ang.max() <= 5.0


def test_mlp_params_roundtrip(T, ctx, net_and_data, tmp_path):
    m, p, X, U = net_and_data
    f = str(tmp_path / "net.bin")
    m.save(f)
    m2 = T.Mlp.load(ctx, f)
    assert m2.K == m.K and np.array_equal(m2.get_params(), m.get_params())
    with pytest.raises(T.TTMError):
        T.Mlp(ctx, 0)


# ----------------------------------------------- order 6, trained network --

NT, R, N = 24, 9.0, 6


@pytest.fixture(scope="module")
def trained(T, ctx):
    """Order-6 field of a seeded 24^3 template; the network is trained on
    (C / ||C||_F, plain maximiser's direction) pairs from every valid voxel of
    one 96^3 tomogram and evaluated on another."""
    tmpl = synth.gaussian_blob_template(NT, seed=7).astype(np.float32)
    p = T.params(order_n=N, mask_radius=R, n_rot_base=256)
    shape = (96, 96, 96)
    M = T.Matcher(ctx, tmpl, p, shape)
    vol, _ = synth.make_tomogram(shape, tmpl, R, 30, 11, snr=0.1, lowpass=True)
    M.run(dev(vol))
    b = M.plan.valid_box()
    zz, yy, xx = np.meshgrid(np.arange(b[0], b[1]), np.arange(b[2], b[3]), np.arange(b[4], b[5]), indexing="ij")
    idx = ((zz * shape[1] + yy) * shape[2] + xx).ravel()
    K = T.ttm_num_components(N)
    dX = torch.empty((idx.size, K), device="cuda")
    dU = torch.empty((idx.size, 3), device="cuda")
    T.ttm_mlp_make_pairs(ctx, M.C, N, M.orient, dev(idx, torch.int64), dX, dU)
    net = T.Mlp(ctx, K, seed=5)
    g = torch.zeros(net.num_params, device="cuda")
    loss0 = net.loss_grad(dX, dU, g) / idx.size
    for ep in range(20):
        net.train(dX, dU, epochs=1, batch=4096, lr=1e-3, seed=100 + ep)
    for ep in range(10):
        net.train(dX, dU, epochs=1, batch=4096, lr=3e-4, seed=200 + ep)
    loss1 = net.loss_grad(dX, dU, g) / idx.size
    # the same schedule in BF16 (tensor-core products, FP32 master weights)
    net16 = T.Mlp(ctx, K, seed=5)
    net16.set_precision(T.TTM_MLP_BF16)
    for ep in range(20):
        net16.train(dX, dU, epochs=1, batch=4096, lr=1e-3, seed=100 + ep)
    for ep in range(10):
        net16.train(dX, dU, epochs=1, batch=4096, lr=3e-4, seed=200 + ep)
    net16.set_precision(T.TTM_MLP_FP32)
    loss1_bf16 = net16.loss_grad(dX, dU, g) / idx.size
    # held-out tomogram, plain and learned maps
    vol2, planted = synth.make_tomogram(shape, tmpl, R, 30, 12, snr=0.1, lowpass=True)
    M.run(dev(vol2))
    sl = torch.empty_like(M.score)
    ol = torch.empty_like(M.orient)
    fl = torch.empty_like(M.frob)
    T.ttm_peak_map(M.plan, M.C, sl, ol, fl, mlp=net)
    torch.cuda.synchronize()
    fb = T.ttm_plan_fallback_count(M.plan)
    sl16 = torch.empty_like(M.score)
    ol16 = torch.empty_like(M.orient)
    T.ttm_peak_map(M.plan, M.C, sl16, ol16, mlp=net16)
    torch.cuda.synchronize()
    return dict(tmpl=tmpl, p=p, M=M, net=net, loss0=loss0, loss1=loss1, sl=sl, ol=ol, fl=fl, fb=fb, box=b,
                centres=planted.centres, vol2=vol2, net16=net16, loss1_bf16=loss1_bf16, sl16=sl16)


def test_training_reduces_loss(trained):
    assert trained["loss1"] < 0.6 * trained["loss0"]


def test_bf16_training_matches_fp32_training(trained):
    """BF16 training (the same initial weights, pairs and schedule) reaches
    the loss of FP32 training to within 10 %, and the learned maximiser with
    the BF16-trained network is also never more than 1e-4 below the plain
    one over every valid voxel."""
    assert trained["loss1_bf16"] < 0.6 * trained["loss0"]
    assert trained["loss1_bf16"] <= 1.1 * trained["loss1"] + 1e-3, (trained["loss1_bf16"], trained["loss1"])
    M, b = trained["M"], trained["box"]
    d = (trained["sl16"] - M.score)[b[0]:b[1], b[2]:b[3], b[4]:b[5]]
    assert int((d < -S_TOL).sum()) == 0


def test_learned_never_below_plain(trained):
    """Error check: over every valid voxel of the held-out tomogram the learned
    score is not more than 1e-4 below the plain maximiser's."""
    M, b = trained["M"], trained["box"]
    d = (trained["sl"] - M.score)[b[0]:b[1], b[2]:b[3], b[4]:b[5]]
    assert int((d < -S_TOL).sum()) == 0
    assert torch.equal(trained["fl"], M.frob)


def test_learned_matches_oracle(trained):
    """Scores within 1e-4 of the oracle (its own field, normaliser and
    direct-sum correlation) at sampled valid voxels and at the planted
    centres. The learned form may return any local maximum within
    the score tolerance of the global one, so orientations are compared
    where the global maximum leads every other local maximum by more than
    that tolerance (and is not flat): at the planted centres and at the
    sampled voxels where this holds."""
    M, b = trained["M"], trained["box"]
    shape = M.score.shape
    zz, yy, xx = np.meshgrid(np.arange(b[0], b[1]), np.arange(b[2], b[3]), np.arange(b[4], b[5]), indexing="ij")
    vi = ((zz * shape[1] + yy) * shape[2] + xx).ravel()
    vi = np.random.default_rng(3).choice(vi, 2000, replace=False)
    inside = [c for c in trained["centres"]
              if b[0] <= c[0] < b[1] and b[2] <= c[1] < b[3] and b[4] <= c[2] < b[5]]
    ci = np.array([(c[0] * shape[1] + c[1]) * shape[2] + c[2] for c in inside], dtype=np.int64)
    assert len(ci) >= 5
    # the oracle's own pipeline: filter, mask, normalised template, field
    # (same quadrature), local normaliser and direct-sum correlation
    pr = O.Prepared(trained["vol2"].astype(np.float64), trained["tmpl"].astype(np.float64), R)
    field = O.tensor_field(pr.tp, O.rotation_set(256), N, 3)
    for idx, min_well in ((vi, 500), (ci, len(ci) // 2)):
        t = dev(idx, torch.int64)
        w, _, _ = O.local_w(pr.g, pr.m, idx, periodic=False, floor=pr.floor)
        Cs = O.correlate(pr.g, field, idx, periodic=False, w=w)
        so, uo, sec, curv = O.maximise(Cs, N, 3, 20000, with_curvature=True)
        sl = trained["sl"].flatten()[t].cpu().numpy()
        ul = trained["ol"].reshape(3, -1)[:, t].cpu().numpy().T
        assert np.abs(sl - so).max() <= S_TOL
        F = O.frobenius(Cs, N)
        well = ((so - sec) > S_TOL) & (curv > 1e-3 * F)
        ang = np.degrees(np.arccos(np.clip(np.abs(np.sum(ul * uo, 1)), 0, 1)))
        assert well.sum() >= min_well
        assert ang[well].max() <= ANG_TOL_DEG


def test_trained_network_start_quality(T, ctx, trained):
    """What the trained network gains over the same network untrained: its
    predicted direction (BF16 tensor-core inference) lies much closer to the
    plain maximiser's orientation on the held-out tomogram. The learned
    maximiser's timing against the plain one is printed (it is not asserted:
    the plain maximiser's tensor-core probe product and angular-suppression
    starts make the network's inference the dearer of the two)."""
    M, b = trained["M"], trained["box"]
    shape = M.score.shape
    zz, yy, xx = np.meshgrid(np.arange(b[0], b[1]), np.arange(b[2], b[3]), np.arange(b[4], b[5]), indexing="ij")
    idx = ((zz * shape[1] + yy) * shape[2] + xx).ravel()
    idx = np.random.default_rng(9).choice(idx, 20000, replace=False)
    K = M.C.shape[0]
    dX = torch.empty((idx.size, K), device="cuda")
    dU = torch.empty((idx.size, 3), device="cuda")
    T.ttm_mlp_make_pairs(ctx, M.C, N, M.orient, dev(idx, torch.int64), dX, dU)
    ustar = dU.cpu().numpy()

    def median_angle(net):
        out = torch.empty_like(dU)
        net.infer(dX, out)
        cos = np.abs(np.sum(out.cpu().numpy() * ustar, 1))
        return float(np.median(np.degrees(np.arccos(np.clip(cos, 0, 1)))))

    a_tr = median_angle(trained["net"])
    a_un = median_angle(T.Mlp(ctx, K, seed=5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2, o2 = torch.empty_like(M.score), torch.empty_like(M.orient)
    times = []
    for kw in ({}, {"mlp": trained["net"]}):
        T.ttm_peak_map(M.plan, M.C, s2, o2, **kw)
        e0.record()
        for _ in range(3):
            T.ttm_peak_map(M.plan, M.C, s2, o2, **kw)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 3)
    print("median angle to u*: trained %.1f deg, untrained %.1f deg; maximiser plain %.2f ms, learned %.2f ms"
          % (a_tr, a_un, times[0], times[1]))
    assert a_tr < 0.5 * a_un


def test_learned_rejects_bad_mlp(T, ctx, trained):
    M = trained["M"]
    wrong = T.Mlp(ctx, 15, seed=1)
    with pytest.raises(T.TTMError):
        T.ttm_peak_map(M.plan, M.C, trained["sl"], trained["ol"], mlp=wrong)
    with pytest.raises(T.TTMError):
        T.ttm_peak_map(M.plan, M.C, trained["sl"], trained["ol"], mode=T.TTM_MAX_MLP_WARM)
