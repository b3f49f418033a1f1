"""Device-side failure detection without a GPU fault: a bounded wait that
nothing completes expires after a short limit, the kernel records the timeout
in the status word and returns, and the host reads RSI_E_TIMEOUT; the device
stays usable afterwards."""
import ctypes

import pytest
import torch

from paper_2408_06765_gb300 import build, rsi
from paper_2408_06765_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RSI_E_TIMEOUT = -3


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def test_expired_wait_is_reported_and_the_context_survives(lib):
    rsi.sync_status()  # clean start
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rsi_selftest_wait_timeout(2_000_000, s) == 0  # ~1 ms at 2 GHz
    assert lib.rsi_sync_status(s) == RSI_E_TIMEOUT
    assert b"expired" in lib.rsi_last_error()
    assert lib.rsi_sync_status(s) == 0  # the word was cleared
    # the context is intact: a chain still runs and checks out clean
    img = rsi.run_chain(W.small_ragged("fp32c", n_piston=300, n_iface=500, nx=8, nz=8)).image
    torch.cuda.synchronize()
    rsi.sync_status()
    assert torch.isfinite(torch.view_as_real(img)).all()


def test_selftest_rejects_bad_limits(lib):
    assert lib.rsi_selftest_wait_timeout(0, None) == -1
