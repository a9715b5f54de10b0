"""Failure detection on the device without a GPU fault: the bounded
mbarrier wait that guards the score kernels' TMA camera staging gives up,
the kernel reports REFINE_ETIMEOUT through the device status word, and the
context stays usable (the copy that the barrier waits for is 16 bytes short,
so its phase can never complete)."""
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
