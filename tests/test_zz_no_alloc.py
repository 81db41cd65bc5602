"""sc_lbm_quad_moments_noalloc: the allocation-free form of the quadrature
moment reduction, called through the C ABI.  It is checked on two calls in a
row against the handle path (sc_lbm_moments) on the same ensemble state and
against the oracle's two-pass moments of the same per-node field, within the
tolerances of the moment tests (mean 1e-12, std 1e-9 absolute).  The first
call carries one non-finite value, which the counter reports and which only
its own cell sees; the second call, on clean data, finds the counter cleared.
A call captured into a CUDA graph is replayed on new field values after the
host weight array was overwritten: the graph keeps the weights it captured.

Named so that pytest collects it last; it passes alone in a fresh process and
after the other tests."""
import numpy as np
import pytest

from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W

torch = pytest.importorskip("torch")


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """Host-side validation: nothing reaches the device, and each message is
    exactly the documented text."""
    n = S.SC_NOALLOC_MAX_NODES + 1
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_quad_moments_noalloc(np.zeros((n, 4)), np.ones(n), None, None)
    assert ei.value.code == S.SC_ERR_SCRATCH
    assert str(ei.value).endswith(": n_nodes = %d exceeds the no-alloc maximum of %d nodes"
                                  % (n, S.SC_NOALLOC_MAX_NODES))
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_quad_moments_noalloc(np.zeros((2, 4)), [1.0, -1.0], None, None)
    assert ei.value.code == S.SC_ERR_ARG
    assert str(ei.value).endswith(": the weights must have a positive finite sum")
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_quad_moments_noalloc(np.zeros((2, 4)), [0.5, 0.5], None, None)
    assert ei.value.code == S.SC_ERR_ARG
    assert str(ei.value).endswith(": null field or output pointer")


def _node_speeds(ens, nq, flags):
    """|u| of every node as the library forms it from its FP32 velocity:
    (ux^2 + uy^2) + uz^2 and the square root, each rounded once in FP32, on
    the host from the exported velocity; solid cells 0.  Host double
    [nq][ncell]."""
    Q = []
    for j in range(nq):
        u = ens.velocity(0, j).cpu().numpy()
        q = np.sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]).astype(np.float64)
        q[flags != 0] = 0.0
        Q.append(q)
    return np.stack(Q)


@pytest.mark.gpu
def test_noalloc_matches_handle_moments_on_two_calls(O):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.URBAN_LES
    cfg = S.make_config(wl)
    _, a = S.sc_lbm_quadrature(cfg, 0)
    flags = S.sc_lbm_geometry(cfg, 0)
    ens = S.Ensemble(cfg)
    stream = torch.cuda.current_stream()
    raw = stream.cuda_stream
    nonfinite = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    k_nan = int(np.flatnonzero(flags == 0)[1000])
    for call, steps in enumerate((60, 40)):   # two calls in a row, on different states
        ens.step(steps)
        ref = ens.moments(0)
        Qh = _node_speeds(ens, len(a), flags)
        Qin = Qh.copy()
        if call == 0:
            Qin[0, k_nan] = np.nan       # one non-finite value, first call only
        Q = torch.from_numpy(Qin).cuda()
        mean = torch.full((Q.shape[1],), float("nan"), dtype=torch.float64, device="cuda")
        std = torch.full_like(mean, float("nan"))
        S.sc_lbm_quad_moments_noalloc(Q, a, mean, std, nonfinite, raw)
        stream.synchronize()
        assert int(nonfinite.item()) == (1 if call == 0 else 0)
        keep = np.ones(Q.shape[1], bool)
        if call == 0:
            keep[k_nan] = False
            assert np.isnan(mean[k_nan].item())
        mg, sg = mean.cpu().numpy()[keep], std.cpu().numpy()[keep]
        assert np.max(np.abs(mg - ref["mean"].cpu().numpy()[keep])) < 1e-12
        assert np.max(np.abs(sg - ref["std"].cpu().numpy()[keep])) < 1e-9
        m_o, s_o, _ = O.moments_two_pass(a, Qh)
        assert np.max(np.abs(mg - m_o[keep])) < 1e-12
        assert np.max(np.abs(sg - s_o[keep])) < 1e-9
        del ref
    ens.close()


@pytest.mark.gpu
def test_noalloc_call_replays_from_a_cuda_graph(O):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(11)
    nq, nc = 9, 3 * 2048 + 37                     # several blocks and a ragged tail
    a = rng.uniform(0.1, 1.0, nq)
    a_captured = a.copy()
    Q = torch.from_numpy(rng.normal(1.0, 0.3, (nq, nc))).cuda()
    mean = torch.empty(nc, dtype=torch.float64, device="cuda")
    std = torch.empty_like(mean)
    nonfinite = torch.zeros(1, dtype=torch.int64, device="cuda")
    # the first call on the device looks up the counter: outside the capture
    S.sc_lbm_quad_moments_noalloc(Q, a, mean, std, nonfinite, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sc_lbm_quad_moments_noalloc(Q, a, mean, std, nonfinite, torch.cuda.current_stream().cuda_stream)
    a[:] = 1.0                                    # the graph must not read the host array again
    for rep in range(2):
        Qh = rng.normal(2.0 + rep, 0.5, (nq, nc))
        keep = np.ones(nc, bool)
        if rep == 1:
            Qh[4, 777] = np.inf
            keep[777] = False
        Q.copy_(torch.from_numpy(Qh))
        g.replay()
        torch.cuda.synchronize()
        assert int(nonfinite.item()) == rep
        m_o, s_o, _ = O.moments_two_pass(a_captured, Qh)
        assert np.max(np.abs(mean.cpu().numpy()[keep] - m_o[keep])) < 1e-12
        assert np.max(np.abs(std.cpu().numpy()[keep] - s_o[keep])) < 1e-9
