"""The continuous-batching server: requests arriving while others run are admitted into the
batch and overlap on the device; every result must equal the same request run alone (within
the solver tolerance), and latencies must be reported."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dg(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return native


@pytest.mark.parametrize("precision", ["mixed64", "fp64"])
def test_served_results_equal_alone(dg, precision):
    from paper_1311_7477_gb300 import serve, workloads
    prec = {"fp64": dg.DG_FP64, "mixed64": dg.DG_MIXED64}[precision]
    trace = workloads.request_trace(count=8, rate=400.0, seed=11, Ns=(16, 24, 32), ns=(2, 3), steps=(3, 14))
    srv = serve.Server(max_active=4, hbm_budget=1e9, precision=prec, precond="twolevel", cg_tol=1e-12, chunk=3,
                       keep_results=True)
    rep = srv.run(trace)
    assert rep["requests"] == len(trace) and rep["batch_status"] == 0
    assert rep["latency_p50_s"] is not None and rep["latency_p99_s"] >= rep["latency_p50_s"]
    # requests overlapped: some were admitted before others finished
    spans = sorted((r.admit_t, r.done_t) for r in srv.done)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for spec in trace:
        g = dg.Grid(spec["N"], spec["N"], spec["n"])
        g.set_precond("twolevel")
        w0 = torch.from_numpy(workloads.initial_field(dg, g, spec)).cuda()
        dt = workloads.stable_dt(dg, spec["N"], spec["n"], spec["D"])
        s = dg.Sim(g, w0, D=spec["D"], dt=dt, precision=prec, cg_tol=1e-12)
        s.step(spec["steps"])
        om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        ps = torch.empty_like(om)
        s.get(om, ps)
        torch.cuda.synchronize()
        wb, pb, nsteps = srv.results[spec["id"]]
        assert nsteps == spec["steps"]
        ew = np.linalg.norm(om.cpu().numpy() - wb) / np.linalg.norm(wb)
        ep = np.linalg.norm(ps.cpu().numpy() - pb) / np.linalg.norm(pb)
        assert ew < 1e-9 and ep < 1e-9, (spec, ew, ep)


def test_failed_request_does_not_stop_the_others(dg):
    """A request whose start-up solve fails (here: a non-finite initial field) ends with its
    error in the report; the other requests are served as usual."""
    from paper_1311_7477_gb300 import serve, workloads
    trace = workloads.request_trace(count=4, rate=400.0, seed=13, Ns=(16, 24), ns=(2, 3), steps=(3, 8))
    bad = trace[1]
    g = dg.Grid(bad["N"], bad["N"], bad["n"])
    w = np.zeros(g.shape)
    w[0, 0, 0, 0] = np.nan
    bad["omega0"] = w
    g.close()
    srv = serve.Server(max_active=4, hbm_budget=1e9, precision=dg.DG_MIXED64, precond="twolevel", cg_tol=1e-10,
                       chunk=3)
    rep = srv.run(trace)
    assert rep["failed"] == 1 and rep["failures"][0]["id"] == bad["id"], rep["failures"]
    assert rep["requests"] == len(trace) - 1 and rep["batch_status"] == 0
    assert sorted(r.id for r in srv.done) == sorted(s["id"] for s in trace if s is not bad)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_request_failing_mid_run_ends_alone(dg, precision):
    """A request whose solves stop converging after admission (its iteration cap cut to one
    iteration once its start-up solve is done) is reported as failed with its error when it
    completes, and left out of the served requests and their latencies; the others are
    served."""
    from paper_1311_7477_gb300 import serve, workloads
    prec = {"fp64": dg.DG_FP64, "mixed": dg.DG_MIXED}[precision]
    trace = workloads.request_trace(count=5, rate=400.0, seed=17, Ns=(16, 24), ns=(2, 3), steps=(6, 12))
    bad = trace[2]
    bad["cg_maxit"] = 1
    srv = serve.Server(max_active=4, hbm_budget=1e9, precision=prec, precond="twolevel", cg_tol=1e-10, chunk=3)
    rep = srv.run(trace)
    assert rep["failed"] == 1 and rep["failures"][0]["id"] == bad["id"], rep["failures"]
    assert "NOCONV" in rep["failures"][0]["error"] or "status 4" in rep["failures"][0]["error"]
    assert rep["requests"] == len(trace) - 1
    assert sorted(r.id for r in srv.done) == sorted(s["id"] for s in trace if s is not bad)
