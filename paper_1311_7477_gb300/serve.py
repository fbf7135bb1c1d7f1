"""Continuous-batching simulation server on one GPU.

Requests (cells per side N, nodes n, viscosity D, number of steps, initial field -- given
as node values in "omega0", or generated from the spec's field recipe by host threads --
and optionally "cg_maxit", the iteration cap of the solves after the start-up one) arrive
over time.  A request is admitted as soon as a batch slot is free and its device-memory
footprint fits the HBM budget; admission builds its simulation (initial Poisson solve) on a
grid shared by all requests of the same (N, n) and takes its two RK4 start-up steps, then
the request joins the batch (dg_batch_admit).  The GPU loop advances every admitted simulation with one persistent,
graph-captured launch per chunk of steps (dg_batch_step); a simulation that has taken all its
steps is retired, its latency (arrival -> completion) recorded and its memory freed, which
admits waiting requests.  Requests that arrive while others are on the GPU therefore overlap
with them on the device.

A request whose simulation reports an error (a solve that did not converge, a non-finite
value, a capped wait) ends alone with that error in the report's "failures" and is left out
of the latency figures and of the throughput; the others are served.  If a mixed-precision
request's start-up solve does not converge, it is admitted once more in float64 ("fallbacks").

All GPU work goes through the C ABI (paper_1311_7477_gb300.dg); this module only decides what
runs when.
"""
import time

import numpy as np

from . import dg, workloads

# device bytes per dof of one simulation (state rings, RK stages, solver and preconditioner
# vectors including the spectral preconditioner's half spectrum, grid workspace), float64 /
# mixed
BYTES_PER_DOF = {dg.DG_FP64: 8 * 24, dg.DG_MIXED: 8 * 24 + 4 * 11, dg.DG_MIXED64: 8 * 24 + 4 * 11,
                 dg.DG_FP64_PC32: 8 * 24 + 4 * 3}


def footprint(N, n, precision):
    return N * N * n * n * BYTES_PER_DOF[precision]


class Request:
    def __init__(self, spec):
        self.spec = spec
        self.id = spec["id"]
        self.arrival = spec["arrival"]
        self.steps = spec["steps"]
        self.admit_t = None
        self.done_t = None
        self.grid = None
        self.sim = None
        self.precision = None
        self.dof_steps = 0        # dof x steps counted for this request so far
        self.remaining = None
        self.field = None
        self.closing = False

    @property
    def dof(self):
        return self.spec["N"] ** 2 * self.spec["n"] ** 2


class Server:
    def __init__(self, max_active=64, hbm_budget=200e9, precision=dg.DG_MIXED, precond="spectral", cg_tol=1e-10,
                 chunk=8, dt_cap=2e-4, keep_results=False, groups=0):
        self.batch = dg.Batch(max_active)
        if groups:
            self.batch.set_groups(groups)
        self.max_active = max_active
        self.budget = float(hbm_budget)
        self.precision = precision
        self.precond = precond
        self.cg_tol = cg_tol
        self.chunk = int(chunk)
        self.dt_cap = dt_cap
        self.keep_results = keep_results
        self.active = []
        self.used = 0.0
        self.done = []
        self.results = {}
        self.dof_steps = 0
        self.grids = {}           # (N, n) -> dg.Grid, shared by the requests of that shape
        self.t = {"field": 0.0, "create": 0.0, "admit": 0.0, "step": 0.0, "finish": 0.0}

    def _grid(self, N, n):
        g = self.grids.get((N, n))
        if g is None:
            g = dg.Grid(N, N, n)
            g.set_precond(self.precond)
            self.grids[(N, n)] = g
        return g

    def _field(self, spec):
        """Host-side initial field of a request (runs in the prefetch threads)."""
        xn, yn = self.nodes[(spec["N"], spec["n"])]
        return workloads.initial_field_from_nodes(xn, yn, spec)

    def _prefetch(self, req):
        s = req.spec
        if s.get("omega0") is not None:        # the request carries its initial field
            from concurrent.futures import Future
            req.field = Future()
            req.field.set_result(s["omega0"])
            return
        key = (s["N"], s["n"])
        if key not in self.nodes:
            g = self._grid(*key)
            xn, yn, _ = g.nodes()
            self.nodes[key] = (xn, yn)
        req.field = self.pool.submit(self._field, s)

    def _admit(self, req, now, clock):
        import torch
        s = req.spec
        t0 = clock()
        g = self._grid(s["N"], s["n"])
        w0 = torch.from_numpy(req.field.result()).cuda()
        req.field = None
        t1 = clock()
        dt = workloads.stable_dt(dg, s["N"], s["n"], s["D"], dt_cap=self.dt_cap)
        req.precision = self.precision
        try:
            sim = dg.Sim(g, w0, D=s["D"], dt=dt, precision=self.precision, cg_tol=self.cg_tol, cg_maxit=100000)
        except dg.DGError as e:
            if e.code != dg.DG_ERR_NOCONV or self.precision == dg.DG_FP64:
                raise
            # the mixed start-up solve did not converge: serve the request in float64
            req.precision = dg.DG_FP64
            sim = dg.Sim(g, w0, D=s["D"], dt=dt, precision=dg.DG_FP64, cg_tol=self.cg_tol, cg_maxit=100000)
            self.fallbacks.append(req.id)
        del w0
        if s.get("cg_maxit"):        # the request's own iteration cap for its later solves
            sim.set_cg(self.cg_tol, int(s["cg_maxit"]))
        t2 = clock()
        req.grid, req.sim = g, sim
        req.admit_t = now
        steps0 = min(2, req.steps)
        if req.steps < 2:
            sim.step(req.steps)
            req.remaining = 0
        else:
            self.batch.set_limit(sim, req.steps)   # batched steps stop at the request's count
            self.batch.admit(sim)          # the two RK4 start-up steps run here
            req.remaining = req.steps - 2
        t3 = clock()
        self.t["field"] += t1 - t0
        self.t["create"] += t2 - t1
        self.t["admit"] += t3 - t2
        self.dof_steps += req.dof * steps0
        req.dof_steps += req.dof * steps0
        self.used += footprint(s["N"], s["n"], req.precision)
        self.active.append(req)

    def _finish(self, req, now, clock=time.perf_counter):
        """The request's last step has completed on the device: check its simulation's status,
        record it (or its failure), keep its result if asked, and free its memory (deferred: a
        free would wait for the running step)."""
        import torch
        t0 = clock()
        req.done_t = now
        # the status is read on a side stream: the legacy stream carries the next batched step
        info = req.sim.status(stream=self.side, check=False)
        failed = info.status != dg.DG_OK
        if failed:
            self.failed.append({"id": req.id, "N": req.spec["N"], "n": req.spec["n"], "error": "status %d after %d "
                                "steps: %s" % (info.status, info.step, dg.lib().dg_last_error().decode())})
            self.dof_steps -= req.dof_steps
        elif self.keep_results:
            om = torch.empty(req.grid.shape, dtype=torch.float64, device="cuda")
            ps = torch.empty_like(om)
            req.sim.get(om, ps)
            torch.cuda.synchronize()
            self.results[req.id] = (om.cpu().numpy(), ps.cpu().numpy(), req.sim.status(check=False).step)
        self.graveyard.append(req.sim)
        req.sim = req.grid = None
        self.used -= footprint(req.spec["N"], req.spec["n"], req.precision)
        self.active.remove(req)
        if not failed:
            self.done.append(req)
        self.t["finish"] += clock() - t0

    def _bury(self):
        for sim in self.graveyard:
            sim.close()
        self.graveyard = []

    def run(self, trace, time_scale=1.0, clock=time.perf_counter):
        """Serves the trace (arrival times scaled by time_scale); returns the report dict.

        One loop: arrivals join the queue and their initial fields are generated by host
        threads; the next batched step is launched as soon as the previous one has been
        queued, so that admissions (host work, then the new simulation's start-up solves on
        the device) overlap the running step; a request whose last step was launched leaves
        the batch at once and completes when that launch's event has fired."""
        import torch
        from concurrent.futures import ThreadPoolExecutor
        pending = sorted((Request(s) for s in trace), key=lambda r: r.arrival)
        queue = []
        inflight = []          # (event, requests whose last step is in that launch)
        self.graveyard = []
        self.failed = []
        self.fallbacks = []
        self.nodes = {}
        self.side = torch.cuda.Stream()
        self.pool = ThreadPoolExecutor(max_workers=4)
        t0 = clock()
        launches = 0
        try:
            while pending or queue or self.active:
                now = clock() - t0
                while pending and pending[0].arrival * time_scale <= now:
                    r = pending.pop(0)
                    self._prefetch(r)
                    queue.append(r)
                # completions
                still = []
                for ev, reqs in inflight:
                    if ev.query():
                        for r in reqs:
                            self._finish(r, clock() - t0, clock)
                    else:
                        still.append((ev, reqs))
                inflight = still
                # admissions by free slots and the HBM budget (FIFO); their host work overlaps
                # the step in flight
                admitted = False
                while queue and len(self.active) < self.max_active:
                    r = queue[0]
                    need = footprint(r.spec["N"], r.spec["n"], self.precision)
                    if self.used + need > self.budget and self.active:
                        break
                    queue.pop(0)
                    try:
                        self._admit(r, clock() - t0, clock)
                    except dg.DGError as e:
                        # a start-up failure (e.g. the initial Poisson solve not converging)
                        # ends this request with its error; the others carry on
                        r.field = None
                        if r.sim is not None:
                            r.sim.close()
                        r.sim = r.grid = None
                        self.failed.append({"id": r.id, "N": r.spec["N"], "n": r.spec["n"],
                                            "error": str(e)})
                        continue
                    admitted = True
                if self.graveyard and admitted:
                    self._bury()   # the admission has synchronised the device: frees do not stall
                # requests with no steps left leave the batch before the next launch; they
                # complete with the work queued so far
                done_now = [r for r in self.active if r.remaining == 0 and not r.closing]
                if done_now:
                    for r in done_now:
                        r.closing = True
                        if r.sim in self.batch.members:
                            self.batch.retire(r.sim)
                    ev = torch.cuda.Event()
                    ev.record()
                    inflight.append((ev, done_now))
                # the next batched step, for every member with steps left
                # (launches of a fixed length: a member whose budget ends inside a launch
                # stops there by its step limit)
                runnable = [r for r in self.active if r.remaining > 0]
                if runnable:
                    k = self.chunk
                    ts = clock()
                    self.batch.step(k)
                    self.t["step"] += clock() - ts
                    launches += 1
                    for r in runnable:
                        taken = min(k, r.remaining)
                        r.remaining -= taken
                        self.dof_steps += r.dof * taken
                        r.dof_steps += r.dof * taken
                if not runnable and not admitted:
                    if inflight:
                        inflight[0][0].synchronize()
                    elif self.graveyard:
                        self._bury()
                    elif pending and not queue:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival * time_scale - (clock() - t0))))
            torch.cuda.synchronize()
            self._bury()
        finally:
            self.pool.shutdown(wait=True)
        wall = clock() - t0
        lat = np.array([r.done_t - r.arrival * time_scale for r in self.done])
        st = self.batch.status(check=False)
        return {"requests": len(self.done), "failed": len(self.failed), "failures": self.failed[:8],
                "fallbacks_fp64": len(self.fallbacks),
                "wall_s": wall,
                "mdof_steps_per_s": self.dof_steps / wall / 1e6,
                "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "batch_launches": launches, "batch_status": st["rc"], "graph": st["graph"],
                "host_seconds": dict(self.t), "grids": len(self.grids)}

    def close(self):
        for g in self.grids.values():
            g.close()
        self.grids = {}
