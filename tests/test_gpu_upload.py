"""State upload through the C ABI: page-locked (pinned, mapped) host memory is read by a
kernel over the host link and narrowed on the way; other memory is copied by the DMA
engines. Both give the same device state, bit for bit, in both precisions, and the direct
path is taken only where the whole buffer lies inside a mapped allocation at a 16-byte
aligned address.
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


def pinned(shape, extra=0):
    import torch
    n = int(np.prod(shape)) + extra
    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_direct_host_read_equals_dma_copy(prec):
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    pr = mw3.Propagator(cfg, precision=prec, tuning={"up_direct": 1})
    pr.propagate(3)
    q, qp = pr.state()
    buf_q, buf_qp = pinned(q.shape), pinned(qp.shape)
    buf_q[:] = q.ravel()
    buf_qp[:] = qp.ravel()
    # pageable copies (DMA engines)
    pr.set_state(np.array(q), np.array(qp))
    assert pr.get_tuning("up_direct_last") == 0
    ref = pr.state()
    # pinned: read directly
    pr.set_state(buf_q.reshape(q.shape), buf_qp.reshape(qp.shape))
    assert pr.get_tuning("up_direct_last") == 1
    got = pr.state()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    # the same pinned memory with the direct path switched off
    pr.set_tuning("up_direct", 0)
    pr.set_state(buf_q.reshape(q.shape), buf_qp.reshape(qp.shape))
    assert pr.get_tuning("up_direct_last") == 0
    for a, b in zip(ref, pr.state()):
        assert np.array_equal(a, b)
    pr.close()


def test_unaligned_pinned_view_falls_back_to_copy():
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    pr = mw3.Propagator(cfg, precision="mixed", tuning={"up_direct": 1})
    pr.propagate(2)
    q, _ = pr.state()
    buf = pinned(q.shape, extra=1)
    view = buf[1:]                      # 8 bytes past a 16-byte boundary
    view[:] = q.ravel()
    pr.set_state(view.reshape(q.shape))
    assert pr.get_tuning("up_direct_last") == 0
    got, _ = pr.state()
    pr.set_state(np.array(q))
    ref, _ = pr.state()
    assert np.array_equal(got, ref)
    pr.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fp32_host_state_equals_fp64_of_the_same_values(prec):
    """mw3_set_state_f32 moves half the bytes; for FP32-representable values it gives the
    same device state as mw3_set_state (mixed: the FP32 state itself; FP64: widened
    exactly)."""
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    pr = mw3.Propagator(cfg, precision=prec)
    pr.propagate(3)
    q, qp = pr.state()
    q32, qp32 = q.astype(np.float32), qp.astype(np.float32)
    pr.set_state(q32.astype(np.float64), qp32.astype(np.float64))
    ref = pr.state()
    pr.set_state_f32(q32, qp32)
    for a, b in zip(ref, pr.state()):
        assert np.array_equal(a, b)
    pr.set_state_f32(q32)                # q_(k-1) = 0
    assert not np.any(pr.state()[1])
    pr.close()
