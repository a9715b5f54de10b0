"""Device self-checks.  Failure detection without a GPU fault: the bounded
mbarrier wait that guards the score kernels' TMA camera staging gives up,
the kernel reports REFINE_ETIMEOUT through the device status word, and the
context stays usable (the copy that the barrier waits for is 16 bytes short,
so its phase can never complete).  Also the FP32 FMA-rate probe that gives
the score kernel's measured roofline denominator."""
import numpy as np
import pytest

from paper_2606_09074_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09074_gb300 import binding as rb
    ctx = rb.Context(0)
    yield torch, rb, ctx
    ctx.close()


def test_bounded_wait_runs_out_and_reports(env):
    torch, rb, ctx = env
    assert ctx.selftest_wait(nbytes=1024, missing=0) == rb.REFINE_OK
    assert ctx.selftest_wait(nbytes=512, missing=16, cycles=2_000_000) == rb.REFINE_ETIMEOUT
    assert "bounded wait" in rb.refine_last_error(ctx.handle).decode()
    assert ctx.selftest_wait(nbytes=16, missing=0) == rb.REFINE_OK  # the status word was cleared
    # the context still scores afterwards
    w = synth.config0(seed=3, n=500, v=4)
    dev = torch.device("cuda", 0)
    s = ctx.score(torch.from_numpy(w.scene.pos).to(dev), torch.from_numpy(w.scene.attr).to(dev),
                  rb.cameras_to_device(w.cams, dev))
    ctx.check()
    assert np.isfinite(s.cpu().numpy()).all()
    for bad in ((8, 0, 1000), (2048, 0, 1000), (1024, 0, 0), (1024, 1 << 20, 1000)):
        assert ctx.selftest_wait(*bad) == rb.REFINE_EINVAL


def test_fma_rate_is_a_plausible_fp32_peak(env):
    """refine_fma_rate measures the FP32 FMA throughput that the score
    kernel's roofline is compared with: it must lie below the nominal peak
    at the part's top clock (2.07 GHz, 2.2 GHz allowed for margin) and well
    above a fifth of it, and it refuses an iteration count out of range."""
    torch, rb, ctx = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.2e9
    rate, ms = ctx.fma_rate(iters=1 << 15)
    assert ms > 0.0
    assert 0.2 * nominal < rate < nominal, (rate, nominal)
    with pytest.raises(rb.RefineError):
        ctx.fma_rate(iters=0)
    with pytest.raises(rb.RefineError):
        ctx.fma_rate(iters=(1 << 20) + 1)
    assert ctx.selftest_wait(nbytes=16, missing=0) == rb.REFINE_OK  # the context is still usable
