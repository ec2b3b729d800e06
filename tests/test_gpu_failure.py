"""Failure detection on the GPU without a fault.

Every mbarrier wait of the tensor-core kernels is bounded. When a wait of the tile-major
angular step runs out, the CTA stops issuing work, waits (with the full bound) for the
tensor-core operations it already committed, frees its tensor memory, sets an error word
and returns; the host reads the word at the chunk boundary and mw3_propagate returns
MW3_ERR_TIMEOUT. The test cuts the bound to zero polls (tuning key tc_wait_limit), so that
every wait runs out while its MMAs are still in flight, and checks the status, and that a
new context on the same device then propagates normally. Nothing traps, faults or hangs.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_expired_tensor_core_wait_returns_timeout():
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    n = 8
    ref = mw3.Propagator(cfg, precision="mixed")
    ref.kernel_times(enable=True)
    ref.propagate(n)
    assert ref.kernel_times()["angular_tc"][1] == n     # the tensor-core angular step ran
    assert ref.get_tuning("tc_wait_limit") == 1 << 22
    q_ref = ref.state()[0].copy()
    ref.close()

    bad = mw3.Propagator(cfg, precision="mixed")
    bad.set_tuning("tc_wait_limit", 0)
    with pytest.raises(mw3.MW3Error) as e:
        bad.propagate(n)
    assert e.value.code == -6                           # MW3_ERR_TIMEOUT
    bad.close()

    again = mw3.Propagator(cfg, precision="mixed")
    again.propagate(n)
    q = again.state()[0]
    np.testing.assert_allclose(q, q_ref, rtol=0, atol=1e-6 * np.max(np.abs(q_ref)))
    again.close()
