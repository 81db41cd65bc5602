"""sc_lbm_quad_moments_noalloc: the allocation-free form of the quadrature
moment reduction, called through the C ABI and checked against the handle
path (sc_lbm_moments) on the same ensemble state, within the tolerances of the
moment tests (mean 1e-12, std 1e-9 absolute), on two calls in a row.

Named so that pytest collects it last; it passes alone in a fresh process and
after the other tests."""
import numpy as np
import pytest

from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W

torch = pytest.importorskip("torch")


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """Host-side validation: nothing reaches the device."""
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_quad_moments_noalloc(np.zeros((S.SC_NOALLOC_MAX_NODES + 1, 4)),
                                      np.ones(S.SC_NOALLOC_MAX_NODES + 1), None, None)
    assert ei.value.code == S.SC_ERR_SCRATCH
    assert "exceeds the no-alloc scratch maximum of %d nodes" % S.SC_NOALLOC_MAX_NODES in str(ei.value)
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_quad_moments_noalloc(np.zeros((2, 4)), [1.0, -1.0], None, None)
    assert ei.value.code == S.SC_ERR_ARG


def _node_speeds(ens, nq):
    """|u| of every node as a device double [nq][ncell] (solid cells 0), and
    the exported velocity tensors, which the caller keeps alive until the
    stream that reads them has finished (they were allocated on the
    handle's stream)."""
    us = [ens.velocity(0, j) for j in range(nq)]
    return torch.stack([torch.linalg.vector_norm(u.double(), dim=0) for u in us]), us


@pytest.mark.gpu
def test_noalloc_matches_handle_moments_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.URBAN_LES
    cfg = S.make_config(wl)
    _, a = S.sc_lbm_quadrature(cfg, 0)
    ens = S.Ensemble(cfg)
    stream = torch.cuda.current_stream()
    raw = stream.cuda_stream
    nonfinite = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    for steps in (60, 40):   # two calls in a row, on different states
        ens.step(steps)
        ref = ens.moments(0)
        Q, us = _node_speeds(ens, len(a))
        mean = torch.full((Q.shape[1],), float("nan"), dtype=torch.float64, device="cuda")
        std = torch.full_like(mean, float("nan"))
        S.sc_lbm_quad_moments_noalloc(Q, a, mean, std, nonfinite, raw)
        stream.synchronize()
        assert int(nonfinite.item()) == 0
        assert torch.max(torch.abs(mean - ref["mean"])).item() < 1e-12
        assert torch.max(torch.abs(std - ref["std"])).item() < 1e-9
        del us, ref
    ens.close()
