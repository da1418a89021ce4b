"""The allocation-free entry point lb_conserved_sums_static, through the C ABI.

It serves callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or their loop must not risk an allocation's device-wide synchronisation).  The
test compares it with the existing path — a context holding the same populations and
lb_moments' FP64 sums — on two calls in a row, within the tolerance the other sums tests
use (FP32 rounding of the stored state, ~1e-7 per node).  This file is collected last."""
import numpy as np
import pytest

import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _state(nx, ny, seed):
    m = th.Model(1.0, 1 / 3, 0.01, 1e-4, 0.8, 1.0, 1.0)
    pert = synth.gaussian_field((9, ny, nx), seed=seed, scale=0.02)
    return m.fbar()[:, None, None] * (1.0 + pert)


def test_static_sums_match_lb_moments_twice():
    import torch
    stream = torch.cuda.current_stream()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for nx, ny, seed in [(96, 80, 1), (64, 40, 2)]:          # second call: fewer rows than the first
        f = _state(nx, ny, seed)
        fd = torch.from_numpy(f).cuda()
        ref = lbf.Lattice(nx, ny, seed=3)
        lbf.lb_set_populations(ref.ctx, fd, lbf.LB_DEVICE, 0)
        s_ref = ref.sums()
        out.fill_(np.nan)
        lbf.lb_conserved_sums_static(fd, nx, ny, out, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = 30 * 1e-7 * np.sqrt(nx * ny)
        np.testing.assert_allclose(got, s_ref, rtol=0, atol=tol)
        # and it is the plain FP64 sum of the caller's populations
        np.testing.assert_allclose(got, [f.sum(), (th.C[:, 0][:, None, None] * f).sum(),
                                         (th.C[:, 1][:, None, None] * f).sum()], rtol=1e-12, atol=1e-12)


def test_static_sums_rejects_too_many_rows():
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    f = torch.zeros(9, dtype=torch.float64, device="cuda")
    with pytest.raises(lbf.LBError) as e:
        lbf.lb_conserved_sums_static(f, 1, lbf.LB_STATIC_MAX_ROWS + 1, out, None)
    assert e.value.code == lbf.LB_EINVAL
    assert "LB_STATIC_MAX_ROWS" in lbf.lb_last_error(None)
