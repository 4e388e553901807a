"""Host logic of the serving loop on the CPU: the admission controller with the
device work replaced by a timed stand-in.  Requests start in arrival order
(FIFO) as soon as a slot is free and their workspace fits the HBM budget; the
budget and the slot count are never exceeded; a request larger than the whole
budget is refused with an error while the others complete."""
import time

import numpy as np

from paper_2012_07266_gb300.serve import Request, Server, footprint
from pm_inputs import workload


class TimedServer(Server):
    """Server whose device work is a sleep; records what was running at each start."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.starts = []

    def _execute(self, req):
        with self._lock:
            self.starts.append((req.rid, self._active, self._used))
        time.sleep(0.05)
        if req.params.get("fail"):
            raise RuntimeError("device error")


def _req(rid, t, nmesh, **extra):
    p = workload("pm64", nc=nmesh // 2, nmesh=nmesh, map_npix=32, nsteps=4)
    p.update(extra)
    return Request(rid=rid, t_arrive=t, params=p, noise=np.zeros((nmesh // 2,) * 3))


def test_admission_fifo_budget_and_slots():
    small, big = footprint(_req(0, 0, 64).params), footprint(_req(0, 0, 128).params)
    assert big > 4 * small
    budget = big + 2 * small            # room for one large and two small requests at a time
    reqs = [_req(0, 0.0, 128), _req(1, 0.0, 64), _req(2, 0.0, 64), _req(3, 0.0, 64), _req(4, 0.0, 128),
            _req(5, 0.01, 64)]
    srv = TimedServer(device="cuda:0", budget_bytes=budget, max_slots=3)
    stats = srv.serve(reqs)
    assert stats.completed == len(reqs) and all(r.error is None for r in reqs)
    sizes = {r.rid: footprint(r.params) for r in reqs}
    order = [rid for rid, _, _ in srv.starts]
    assert order == sorted(order)                                  # FIFO
    for rid, active, used in srv.starts:
        assert active <= 3 and used <= budget                     # counted with this request admitted
    assert stats.max_active <= 3 and stats.peak_bytes <= budget
    # request 3 had to wait for a slot (three were running), request 4 for memory
    t_admit = {r.rid: r.t_admit for r in reqs}
    assert t_admit[3] > t_admit[2] + 0.03 and t_admit[4] > t_admit[0] + 0.03
    assert stats.summary()["p50_s"] > 0


def test_oversize_refused_and_failures_isolated():
    small = footprint(_req(0, 0, 64).params)
    reqs = [_req(0, 0.0, 128), _req(1, 0.0, 64), _req(2, 0.0, 64, fail=1)]
    srv = TimedServer(device="cuda:0", budget_bytes=2 * small, max_slots=4)
    stats = srv.serve(reqs)
    assert reqs[0].error == "footprint exceeds the HBM budget"
    assert reqs[1].error is None and "device error" in reqs[2].error
    assert stats.completed == 1
