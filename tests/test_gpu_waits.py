"""Bounded device waits (failure detection without a GPU fault): the
TMA-staged fused z pass waits on its copies with a poll limit; when a wait
expires the kernel records it and returns, and the host reads the record
as TTM_E_TIMEOUT. A limit of 0 makes every such wait expire at once, so the
error path runs without anything hanging; the context stays usable."""
import numpy as np
import pytest

from paper_2408_02398_gb300 import synth

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


def test_expired_wait_is_reported_and_context_recovers(T):
    ctx = T.Context(0)
    shape = (64, 64, 64)          # z length 64 (register four-step), 64 * 33 columns: the TMA path
    tmpl = synth.gaussian_blob_template(16, seed=4).astype(np.float32)
    p = T.params(order_n=2, mask_radius=7.0, n_rot_base=16)
    m = T.Matcher(ctx, tmpl, p, shape)
    tomo = torch.as_tensor(synth.normals(8, 1, int(np.prod(shape))).reshape(shape).astype(np.float32), device="cuda")
    T.ttm_correlate(m.plan, tomo, m.C)
    T.ttm_ctx_device_status(ctx)                 # nothing expired
    ref = m.C.clone()
    assert float(ref.abs().max()) > 0
    T.ttm_ctx_set_wait_limit(ctx, 0)
    m.C.fill_(7.0)
    T.ttm_correlate(m.plan, tomo, m.C)           # every bounded wait expires at once
    with pytest.raises(T.TTMError) as e:
        T.ttm_ctx_device_status(ctx)
    assert e.value.code == 6                     # TTM_E_TIMEOUT
    T.ttm_ctx_device_status(ctx)                 # the record was cleared
    T.ttm_ctx_set_wait_limit(ctx, 1 << 22)
    T.ttm_correlate(m.plan, tomo, m.C)
    T.ttm_ctx_device_status(ctx)
    assert torch.equal(m.C, ref)
    with pytest.raises(T.TTMError):
        T.ttm_ctx_set_wait_limit(ctx, -1)
