"""The bench's per-phase breakdown on the host: a forest double that records
calls stands in for the library, so the arithmetic (milliseconds per step,
the ghost rounds' share, host phases left out) and the call order (tracing
on, one untimed step, totals cleared, the traced steps, tracing off) are
checked without a GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PHASES = ("ghost_r1", "ghost_r2", "stage", "fluxfix", "dt", "conserved", "flags", "transfer", "mesh_host",
          "pattern_host")


class FakeForest:
    def __init__(self, totals):
        self.calls = []
        self.totals = totals

    def trace(self, on=True):
        self.calls.append(("trace", on))

    def step(self, n, gather=False, stream=None, scheme="heun"):
        self.calls.append(("step", n, gather, scheme))

    def trace_read(self, reset=True):
        self.calls.append(("read", reset))
        out = {p: (0.0, 0) for p in PHASES}
        if sum(1 for c in self.calls if c[0] == "read") == 2:
            out.update(self.totals)
        return out


def test_phase_breakdown_arithmetic_and_call_order():
    f = FakeForest({"ghost_r1": (1.0, 4), "ghost_r2": (0.6, 4), "stage": (6.0, 4), "dt": (0.4, 2),
                    "mesh_host": (100.0, 1)})
    r = bench.phase_breakdown(f, None, True, steps=2, scheme="ssp3")
    assert r["ms_per_step"] == {"ghost_r1": 0.5, "ghost_r2": 0.3, "stage": 3.0, "dt": 0.2}
    assert abs(r["ghost_share"] - 0.8 / 4.0) < 1e-12
    assert r["gather"] is True and r["steps"] == 2
    assert f.calls == [("trace", True), ("step", 1, True, "ssp3"), ("read", True), ("step", 2, True, "ssp3"),
                       ("read", True), ("trace", False)]


def test_phase_breakdown_without_ghost_rounds():
    f = FakeForest({"stage": (2.0, 4), "dt": (0.02, 2)})
    r = bench.phase_breakdown(f, None, True)
    assert r["ghost_share"] == 0.0 and set(r["ms_per_step"]) == {"stage", "dt"}
