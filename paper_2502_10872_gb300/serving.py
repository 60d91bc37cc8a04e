"""Continuous-batching request loop over the C-ABI batch (argument marshalling and scheduling only).

Requests (meshes with a step count) arrive over time. A request is admitted as soon as the batch's HBM
budget holds its instance: its handle is created (host topology, multigrid set-up, the GPU precompute and
assembly) on one of a few worker threads while the GPU steps the resident instances, then it joins the
batch between two steps. Set-up is mostly host work, so several requests are built at once. Every
step advances all resident instances in one persistent launch. A request retires
(and frees its device memory) after its last step. Each instance's result does not depend on the others
in the batch (deterministic, team-size independent reductions), so a request gives the same state alone or
in any mix.

Reported: aggregate vertex-steps/s over the wall time, per-step device latency p50/p99 of the batch, the
queueing delay (arrival to admission) and per-request completion times.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque
from typing import Callable, List, Optional

import numpy as np

from . import binding as gb


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    scenario: object            # anything create_from_scenario accepts
    steps: int
    handle: Optional[gb.Handle] = None
    slot: int = -1
    done_steps: int = 0
    admitted_s: float = float("nan")
    finished_s: float = float("nan")
    status: int = 0
    final_state: Optional[tuple] = None


@dataclasses.dataclass
class ServeReport:
    wall_s: float
    vertex_steps: int
    steps: int
    step_ms: np.ndarray
    requests: List[Request]

    @property
    def vertex_steps_per_s(self) -> float:
        return self.vertex_steps / self.wall_s if self.wall_s > 0 else 0.0

    def summary(self) -> dict:
        lat = self.step_ms
        q = [r.admitted_s - r.arrival_s for r in self.requests if np.isfinite(r.admitted_s)]
        return {
            "requests": len(self.requests),
            "completed": sum(1 for r in self.requests if np.isfinite(r.finished_s)),
            "failed": sum(1 for r in self.requests if r.status != 0),
            "batch_steps": self.steps,
            "vertex_steps": self.vertex_steps,
            "vertex_steps_per_s": self.vertex_steps_per_s,
            "wall_s": self.wall_s,
            "step_ms_p50": float(np.percentile(lat, 50)) if len(lat) else None,
            "step_ms_p99": float(np.percentile(lat, 99)) if len(lat) else None,
            "queue_s_p50": float(np.percentile(q, 50)) if q else None,
            "queue_s_p99": float(np.percentile(q, 99)) if q else None,
        }


class Server:
    """Admit requests into one batch by an HBM budget and step them together."""

    # Launch shape of the batch's step kernel (CTAs per SM, CTA-share scale, clusters), measured on the
    # serving mix (1k-250k-vertex requests): the 5-CTA-per-SM variant with a small share scale, so that the
    # largest resident requests get large teams. Serving, 10 s on one box: the library's default (3 CTAs per
    # SM, share 1) 134.8 M vertex-steps/s; (5, 2.0), the shape the autotuner picks for batches of instances
    # of at most 66 row blocks, 51.8-56.3 M; (5, 1.0) 131.1 M; (5, 0.5) 186.3 M; (5, 0.25) 203.7-205.4 M;
    # (5, 0.125) 211.6 M; (5, 0.0625) 208.8 M. None keeps the library's default.
    DEFAULT_LAUNCH = (5, 0.125, False)

    def __init__(self, budget_bytes: int, precision: str = "fp32_refine", keep_states: bool = False,
                 create_kw: Optional[dict] = None, clock: Callable[[], float] = time.perf_counter,
                 n_workers: int = 4, launch: Optional[tuple] = DEFAULT_LAUNCH):
        self.budget = int(budget_bytes)
        self.n_workers = max(1, int(n_workers))
        self.device = None
        try:
            import torch
            if torch.cuda.is_available():
                self.device = torch.cuda.current_device()
        except Exception:
            pass
        self.precision = precision
        self.keep_states = keep_states
        self.create_kw = create_kw or {}
        self.clock = clock
        self.batch = gb.shell_batch_create(self.budget)
        if launch is not None:
            gb.shell_batch_set_launch(self.batch, *launch)
        self.used = 0

    def _create(self, req: Request):
        if self.device is not None:   # the CUDA device is per thread
            import torch
            torch.cuda.set_device(self.device)
        req.handle = gb.create_from_scenario(req.scenario, precision=self.precision, **self.create_kw)

    def run(self, requests: List[Request], max_wall_s: float = 1e9, steps_per_launch: int = 1) -> ServeReport:
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        ready: deque = deque()          # created handles waiting for budget
        active: dict = {}               # slot -> request
        lat: list = []
        vsteps = 0
        nsteps = 0
        t0 = self.clock()
        building: list = []             # (thread, request) being created

        def now():
            return self.clock() - t0

        while pending or ready or active or building:
            if now() > max_wall_s:
                break
            # start building arrived requests on worker threads (overlaps the GPU step)
            while len(building) < self.n_workers and pending and pending[0].arrival_s <= now():
                req = pending.popleft()
                th = threading.Thread(target=self._create, args=(req,))
                th.start()
                building.append((th, req))
            still = []
            for th, req in building:
                if th.is_alive():
                    still.append((th, req))
                else:
                    th.join()
                    if req.handle is None:
                        raise RuntimeError(f"request {req.rid}: shell_create failed on its worker thread")
                    ready.append(req)
            building = still
            # admit what fits the budget
            while ready:
                req = ready[0]
                rc = gb.shell_batch_admit(self.batch, req.handle, check=False)
                if isinstance(rc, int) and rc == gb.SHELL_ERR_BUDGET:
                    break
                if isinstance(rc, int) and rc < 0:
                    raise gb.ShellError(rc, "shell_batch_admit")
                req.slot = rc
                req.admitted_s = now()
                active[req.slot] = req
                ready.popleft()
            if not active:
                if building:
                    building[0][0].join(timeout=0.001)
                elif pending:
                    time.sleep(min(0.001, max(0.0, pending[0].arrival_s - now())))
                continue
            # one batch step for every resident instance
            n = steps_per_launch
            rc, stats = gb.shell_batch_step(self.batch, n, check=False)
            lat.extend(gb.shell_batch_step_times(self.batch, n).tolist())
            nsteps += n
            for slot, req in list(active.items()):
                st = stats.raw(slot)
                if st is None:
                    continue
                req.done_steps += st.steps_done
                vsteps += st.steps_done * req.scenario.n_verts
                if st.status != 0:
                    req.status = st.status
                if req.done_steps >= req.steps or req.status != 0:
                    req.finished_s = now()
                    if self.keep_states:
                        req.final_state = gb.shell_get_state(req.handle)
                    gb.shell_batch_retire(self.batch, slot)
                    gb.shell_destroy(req.handle)
                    req.handle = None
                    del active[slot]
        wall = now()
        for th, req in building:
            th.join()
            if req.handle is not None:   # built after the wall limit: never admitted
                gb.shell_destroy(req.handle)
                req.handle = None
        return ServeReport(wall, vsteps, nsteps, np.asarray(lat, np.float64), list(requests))

    def close(self):
        if self.batch is not None:
            gb.shell_batch_destroy(self.batch)
            self.batch = None
