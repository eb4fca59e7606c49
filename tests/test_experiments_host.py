"""Host logic of the storage-precision comparison driver (CPU only): a stand-in for the
simulation handle records what the driver asks of it, so the bookkeeping (records every
`every` steps, identical wires in every run, a run that latches a failure stopping at the
next record and still being measured there) is checked without a GPU."""
import numpy as np

from paper_2607_06794_b300 import Config, experiments
from paper_2607_06794_b300.workloads import Workload


class FakeSim:
    """Steps advance a counter; status latches `fail_code` once `fail_at` steps have run."""
    made = []

    def __init__(self, cfgs, fail_at=None, fail_code=6):
        self.cfgs, self.done, self.err = cfgs, 0, 0
        self.fail_at, self.fail_code = fail_at, fail_code
        self.cleared, self.closed, self.wires = 0, False, {}
        FakeSim.made.append(self)

    def set_substrate_pattern(self, k, th):
        pass

    def add_nanowires(self, k, n, length, cen, dirs):
        self.wires[k] = (n, length, np.array(cen), np.array(dirs))

    def step(self, n):
        self.done += n
        if self.fail_at is not None and self.done >= self.fail_at:
            self.err = self.fail_code

    def status(self):
        return self.err

    def clear_error(self):
        self.err = 0
        self.cleared += 1

    def sync(self):
        if self.err:
            raise RuntimeError("latched")

    def shape(self, k):
        return {"volume": 100.0 - self.done, "height": 1.0}

    def descriptors(self, k):
        return {"S_x": 0.1 * k, "n_clusters": 1, "percolates": 0, "step": self.done}

    def close(self):
        self.closed = True


def _workload(prec):
    return Workload("fake", [Config(16, 16, 8, prec=prec), Config(16, 16, 8, prec=prec)],
                    [None, None], [(2, 4.0), (2, 4.0)], 100)


def _wires():
    cen = np.array([[4.0, 4.0, 2.0], [10.0, 10.0, 2.0]])
    dirs = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    return [(cen, dirs, 2), (cen + 1.0, dirs, 2)]


def test_every_run_records_every_instance_with_the_same_wires(monkeypatch):
    FakeSim.made = []
    monkeypatch.setattr(experiments, "Simulation", lambda cfgs: FakeSim(cfgs))
    res = experiments.storage_comparison(_workload, ("fp64", "fp16"), steps=50, every=20, wires=_wires())
    assert set(res) == {"fp64", "fp16"}
    for prec, r in res.items():
        assert r["status"] == 0 and r["stopped_at"] is None
        steps = [e["step"] for e in r["series"]]
        assert steps == [0, 20, 40, 50]
        assert len(r["instances"]) == 2
        assert [i["descriptors"]["S_x"] for i in r["instances"]] == [0.0, 0.1]
    a, b = FakeSim.made
    for k in (0, 1):
        assert np.array_equal(a.wires[k][2], b.wires[k][2]) and a.wires[k][0] == 2
    assert a.closed and b.closed


def test_a_run_that_latches_a_failure_stops_and_is_measured_where_it_stopped(monkeypatch):
    FakeSim.made = []
    monkeypatch.setattr(experiments, "Simulation", lambda cfgs: FakeSim(cfgs, fail_at=35))
    res = experiments.storage_comparison(_workload, ("fp32",), steps=100, every=10, wires=_wires())
    r = res["fp32"]
    assert r["status"] == 6 and r["stopped_at"] == 40  # noticed at the first record after it
    assert r["series"][-1]["step"] == 40 and r["final"]["volume"] == 60.0
    assert r["descriptors"] is not None and r["descriptors"]["step"] == 40
    assert FakeSim.made[0].cleared == 1
