"""Batched persistent stepping (dg_batch): uneven simulations -- different cell counts, n,
viscosities, precisions and preconditioners -- advanced together by one persistent kernel
must give what each gives when stepped alone."""
import numpy as np
import pytest

from paper_1311_7477_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dg(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return native


SPECS = [  # (N, n, D, precision, precond, seed)
    (32, 2, 1e-3, "fp64", "twolevel", 1),
    (24, 3, 0.0, "fp64", "jacobi", 2),
    (16, 5, 5e-4, "fp64", "twolevel", 3),
    (40, 4, 2e-4, "mixed64", "twolevel", 4),
    (20, 3, 1e-3, "mixed", "twolevel", 5),
    (8, 1, 0.0, "fp64", "jacobi", 6),
    (32, 4, 1e-4, "fp64", "spectral", 7),
    (12, 3, 0.0, "mixed", "spectral", 8),
]


def _make(dg, N, n, D, prec, pc, seed, fixed):
    g = dg.Grid(N, N, n)
    g.set_precond(pc)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = torch.from_numpy(fields.random_phase(X, Y, seed=seed, kmax=4)).cuda()
    P = {"fp64": dg.DG_FP64, "mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[prec]
    s = dg.Sim(g, w0, D=D, dt=2e-3, precision=P, cg_tol=1e-12)
    if fixed and prec == "fp64" and g.dof >= 2000:
        # the exact (spectral) preconditioner solves in one iteration; more would iterate on noise
        s.set_cg(1e-30, 1000, fixed_iters=1 if pc == "spectral" else 10)
    return g, s


def _state(g, s):
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    s.get(om, ps)
    torch.cuda.synchronize()
    return om.cpu().numpy(), ps.cpu().numpy()


@pytest.mark.parametrize("groups", [0, 1, 3])
def test_batch_matches_alone(dg, groups):
    alone = [_make(dg, *spec, fixed=True) for spec in SPECS]
    mixed = [_make(dg, *spec, fixed=True) for spec in SPECS]
    b = dg.Batch(16)
    if groups:
        b.set_groups(groups)
    for g, s in mixed:
        b.admit(s)                      # takes the two RK4 start-up steps alone
    b.step(3)
    b.step(3)
    st = b.status()
    assert st["rc"] == 0 and st["launches"] == 2
    for (g, s) in alone:
        s.step(8)
    for spec, (ga, sa), (gb, sb) in zip(SPECS, alone, mixed):
        wa, pa = _state(ga, sa)
        wb, pb = _state(gb, sb)
        ew = np.linalg.norm(wa - wb) / np.linalg.norm(wa)
        ep = np.linalg.norm(pa - pb) / np.linalg.norm(pa)
        # float64 members with >= 2000 dof run the same fixed CG iterations: rounding-order
        # level; members with a tolerance-stopped solve agree to the solver tolerance
        tol = 1e-12 if (spec[3] == "fp64" and gb.dof >= 2000) else 1e-8
        assert ew < tol and ep < tol, (spec, ew, ep)
        assert sb.status().step == 8


def test_batch_graph_retire_readmit(dg):
    members = [_make(dg, *spec, fixed=False) for spec in SPECS[:4]]
    ref = [_make(dg, *spec, fixed=False) for spec in SPECS[:4]]
    b = dg.Batch(8)
    for g, s in members:
        b.admit(s)
    for _ in range(3):                  # the third launch of an unchanged plan is a graph
        b.step(1)
    st = b.status()
    assert st["graph"], "no CUDA graph: " + dg.lib().dg_last_error().decode()
    g0, s0 = members[0]
    b.retire(s0)
    s0.step(1)                          # alone between batch steps
    b.admit(s0)
    b.step(2)
    # 2 RK4 start-up steps at admission, 3 + 2 batched; the retired member one more alone
    expect = [8] + [7] * (len(members) - 1)
    for (g, s), k in zip(ref, expect):
        s.step(k)
    for (ga, sa), (gb, sb), k in zip(ref, members, expect):
        wa, _ = _state(ga, sa)
        wb, _ = _state(gb, sb)
        assert np.linalg.norm(wa - wb) / np.linalg.norm(wa) < 1e-8
        assert sb.status().step == k


def test_batch_step_limits(dg):
    """Members with different step budgets share launches of a fixed length: each stops at
    its limit (dg_batch_set_limit) and matches the same number of steps taken alone."""
    specs = SPECS[:3]
    limits = [4, 7, 0]                  # step indices; 0: no limit
    members = [_make(dg, *spec, fixed=False) for spec in specs]
    ref = [_make(dg, *spec, fixed=False) for spec in specs]
    b = dg.Batch(8)
    for (g, s), lim in zip(members, limits):
        b.set_limit(s, lim)
        b.admit(s)
    b.step(3)
    b.step(3)                           # 2 start-up + 6 batched, unless limited
    expect = [4, 7, 8]
    for (g, s), k in zip(ref, expect):
        s.step(k)
    for (ga, sa), (gb, sb), k in zip(ref, members, expect):
        assert sb.status().step == k
        wa, _ = _state(ga, sa)
        wb, _ = _state(gb, sb)
        assert np.linalg.norm(wa - wb) / np.linalg.norm(wa) < 1e-8
    with pytest.raises(RuntimeError):
        b.set_limit(members[0][1], -1)


def test_batch_autotune(dg):
    """dg_batch_autotune times candidate launch configurations on the live batch (groups, per-n
    tiles, blocks per SM) and keeps the fastest; the members then still match the same steps
    taken alone, a second call for the same member classes is a cache hit, and explicit tiles
    that do not fit are rejected at the next step."""
    import time
    members = [_make(dg, *spec, fixed=False) for spec in SPECS]
    ref = [_make(dg, *spec, fixed=False) for spec in SPECS]
    b = dg.Batch(8)
    for g, s in members:
        b.admit(s)
    cfg = b.autotune(trial_steps=1)
    assert cfg.startswith("groups=") and " n5:" in cfg, cfg
    steps = members[0][1].status().step
    assert all(s.status().step == steps for _, s in members) and steps > 10
    t0 = time.perf_counter()
    assert b.autotune(trial_steps=1) == cfg                 # cached: the same member classes
    assert time.perf_counter() - t0 < 0.5
    assert members[0][1].status().step == steps
    b.step(2)
    for (g, s) in ref:
        s.step(steps + 2)
    for (ga, sa), (gb, sb) in zip(ref, members):
        wa, _ = _state(ga, sa)
        wb, _ = _state(gb, sb)
        assert np.linalg.norm(wa - wb) / np.linalg.norm(wa) < 1e-8
    assert b.status()["rc"] == 0
    b.set_tiles(5, rhs=(32, 32))                            # ~1 MB of shared memory per block
    with pytest.raises(dg.DGError):
        b.step(1)
    b.set_tiles(5)
    b.step(1)
