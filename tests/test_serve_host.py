"""Host logic of the serving loop (paper_2605_18254_gb300/serve.py) on the
CPU: pools are replaced by fakes that finish a job after a set number of
advances, so admission order, pool choice by capacity and dimension,
slot reuse, the read-back of every finished job, the time limit and the
summaries are checked without a GPU."""
import dataclasses

import numpy as np
import pytest

from paper_2605_18254_gb300 import serve


@dataclasses.dataclass
class FakeJob:
    dim: int
    n: int
    cells: int
    work: int  # advances until done


class FakePool:
    def __init__(self, slots):
        self.jobs = {}
        self.log = []
        self.slots = slots

    def admit(self, s, job):
        assert s not in self.jobs and 0 <= s < self.slots
        self.jobs[s] = [job[0], 0]
        self.log.append(("admit", s, job[0].n))

    def advance(self, k):
        for v in self.jobs.values():
            v[1] += 1

    def poll(self):
        return [s for s, (j, w) in self.jobs.items() if w >= j.work]

    def certify(self, s):
        return (0, 0.1, 0.5)

    def state(self, s):
        return {"sweeps": 7}

    def positions(self, s):
        self.log.append(("read", s))
        return np.zeros((self.jobs[s][0].n, self.jobs[s][0].dim)), np.zeros(self.jobs[s][0].n)

    def release(self, s):
        self.log.append(("release", s))
        del self.jobs[s]

    def close(self):
        pass


def make_server(specs):
    srv = serve.Server.__new__(serve.Server)
    srv.specs = list(specs)
    srv.pools = [FakePool(p.slots) for p in specs]
    srv.free = [list(range(p.slots)) for p in specs]
    srv.running = [dict() for _ in specs]
    srv.advance = 1
    srv.keep_results = False
    return srv


@pytest.fixture(autouse=True)
def fake_footprint(monkeypatch):
    monkeypatch.setattr(serve, "srm_job_footprint", lambda job: (job.n, job.cells))


def req(rid, arrival, dim, n, cells, work):
    return serve.Request(rid=rid, arrival=arrival, job=(FakeJob(dim, n, cells, work), None))


def test_admission_by_capacity_and_dimension():
    specs = [serve.PoolSpec(slots=1, max_particles=100, max_cells=50, dim=2),
             serve.PoolSpec(slots=1, max_particles=100, max_cells=50, dim=3),
             serve.PoolSpec(slots=1, max_particles=10_000, max_cells=5000, dim=0)]
    srv = make_server(specs)
    reqs = [req(0, 0.0, 2, 50, 10, 3), req(1, 0.0, 3, 60, 10, 2), req(2, 0.0, 3, 5000, 400, 1),
            req(3, 0.0, 2, 80, 20, 1)]
    done, wall = srv.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    pool = {r.rid: r.pool for r in done}
    assert pool[0] == 0 and pool[1] == 1 and pool[2] == 2
    # request 3 (2D, small) waits for the 2D slot, or takes the big any-dimension slot when free
    assert pool[3] in (0, 2)
    for r in done:
        assert r.certified == (0, 0.1, 0.5) and r.sweeps == 7
        assert r.admitted <= r.finished
    # every finished job was read back before its slot was released
    for p in srv.pools:
        for i, ev in enumerate(p.log):
            if ev[0] == "release":
                assert p.log[i - 1] == ("read", ev[1])


def test_first_come_first_served_and_slot_reuse():
    specs = [serve.PoolSpec(slots=2, max_particles=100, max_cells=50)]
    srv = make_server(specs)
    reqs = [req(i, 0.0, 3, 10 + i, 5, 2 + i % 3) for i in range(7)]
    done, _ = srv.run(reqs)
    admits = [e for e in srv.pools[0].log if e[0] == "admit"]
    assert [e[2] for e in admits] == [10 + i for i in range(7)]  # arrival order
    assert {e[1] for e in admits} == {0, 1}  # two slots reused
    assert srv.free[0] and sorted(srv.free[0]) == [0, 1]


def test_request_fitting_no_pool_is_refused():
    srv = make_server([serve.PoolSpec(slots=1, max_particles=100, max_cells=50, dim=2)])
    with pytest.raises(ValueError):
        srv.run([req(0, 0.0, 3, 10, 5, 1)])
    with pytest.raises(ValueError):
        srv.run([req(1, 0.0, 2, 1000, 5, 1)])


def test_time_limit():
    srv = make_server([serve.PoolSpec(slots=1, max_particles=100, max_cells=50)])
    with pytest.raises(TimeoutError):
        srv.run([req(0, 0.0, 3, 10, 5, 10 ** 9)], time_limit=0.05)


def test_summary_and_poisson_stream():
    a = serve.poisson_stream(200, 5.0, 3, lambda i, rng: (FakeJob(3, 10, 5, 1), None))
    b = serve.poisson_stream(200, 5.0, 3, lambda i, rng: (FakeJob(3, 10, 5, 1), None))
    t = np.array([r.arrival for r in a])
    assert np.array_equal(t, [r.arrival for r in b])  # seeded
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.2) < 0.05  # mean inter-arrival 1 / rate
    done = []
    for i in range(100):
        r = req(i, 0.0, 3, 100, 5, 1)
        r.particles, r.admitted, r.finished, r.sweeps, r.certified = 100, 0.5, 1.0 + i / 100, 10, (0, 0.1, 0.5)
        done.append(r)
    s = serve.summarize(done, 4.0)
    assert s["jobs"] == 100 and s["all_certified"]
    assert s["particle_updates_per_s"] == pytest.approx(100 * 100 * 10 / 4.0)
    assert s["time_to_target_p50_s"] == pytest.approx(np.percentile([1.0 + i / 100 for i in range(100)], 50))
    assert s["service_p99_s"] == pytest.approx(np.percentile([0.5 + i / 100 for i in range(100)], 99))
