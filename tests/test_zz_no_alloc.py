"""The allocation-free entry point mw3_norms_noalloc, checked against the norms the
regular propagation reports (mw3_norm_trace).

It serves callers that cannot call cudaMalloc (a fixed arena, a no-allocation region):
its scratch is a static device array, so these tests hand it device buffers made up
front and compare, on two calls in a row, with the norm of the same state computed by
the context's own kernels. This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_noalloc_norms_match_propagation_norms(torch):
    from paper_2412_10167_gb300 import mw3
    cfg = W.C3_SMALL                      # 3 J values, uneven helicity stacks, 2 states
    pr = mw3.Propagator(cfg, precision="fp64")
    pr.propagate(37)
    ref = pr.norm_trace()[-1]             # ||q_37||^2 per J from the context's kernels
    q, _ = pr.state()                     # the same state as grid values
    nblk, npb = q.shape[0], int(np.prod(q.shape[1:]))
    x = torch.from_numpy(q.reshape(-1)).to("cuda")
    out = torch.zeros(nblk, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    from oracle.hamiltonian import GridHamiltonian
    bj = GridHamiltonian(cfg).block_J_index()
    for call in range(2):                 # two calls in a row share the static scratch
        out.fill_(-1.0)
        mw3.mw3_norms_noalloc(x.data_ptr(), npb, nblk, out.data_ptr(), stream)
        torch.cuda.synchronize()
        per_block = out.cpu().numpy()
        per_J = np.array([per_block[bj == i].sum() for i in range(len(cfg["J"]))])
        np.testing.assert_allclose(per_J, ref, rtol=1e-12)
    # one segment: the whole vector
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    mw3.mw3_norms_noalloc(x.data_ptr(), nblk * npb, 1, tot.data_ptr(), stream)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tot.item(), ref.sum(), rtol=1e-12)
    pr.close()


def test_noalloc_rejects_sizes_beyond_capacity(torch):
    from paper_2412_10167_gb300 import mw3
    x = torch.ones(65 * 8, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    for nseg in (0, 65):
        with pytest.raises(mw3.MW3Error) as e:
            mw3.mw3_norms_noalloc(x.data_ptr(), 8, nseg, out.data_ptr())
        assert e.value.code == -1
    mw3.mw3_norms_noalloc(x.data_ptr(), 8, 64, out.data_ptr())
    torch.cuda.synchronize()
    assert np.all(out[:64].cpu().numpy() == 8.0)
