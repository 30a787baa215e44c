"""Host logic of bench.py's added legs on CPU, with the device work replaced by stand-ins:
the iteration sweep's line through the frame times, and a failing leg reported in its
output instead of ending the bench line."""
import numpy as np

import bench


class _Frame:
    """A stand-in instance whose frame costs 60 us plus 37 us per iteration."""

    def __init__(self, wl, precision=32, graph=True):
        self.iters = wl["params"]["iters"]
        self.n_act = 4

    def update_params(self, iters=None):
        self.iters = iters

    def frame_launches(self):
        return 6 + 6 * self.iters

    def close(self):
        pass


def _patch(monkeypatch, frame_ms):
    import paper_2202_11945_gb300 as pkg
    import torch
    monkeypatch.setattr(pkg, "Reconstructor", _Frame)
    monkeypatch.setattr(bench, "time_frames", lambda R, S, steps, warmup, flush, dm: frame_ms(R, steps))
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: real_empty(*a, **{x: y for x, y in k.items() if x != "device"}))


def test_iteration_sweep_fits_the_per_iteration_cost(monkeypatch):
    _patch(monkeypatch, lambda R, steps: np.full(steps, 0.060 + 0.037 * R.iters))
    out = bench.time_iteration_sweep({"name": "w", "params": {"iters": 4}}, None, None, 50)
    assert "error" not in out
    assert abs(out["us_per_iteration"] - 37.0) < 1e-6 and abs(out["us_fixed"] - 60.0) < 1e-6
    assert out["max_rel_deviation_from_line"] < 1e-9
    assert out["iters4"]["launches_per_frame"] == 30
    assert abs(out["iters1"]["frames_per_s"] - 1e3 / 0.097) < 1e-6


def test_a_failing_leg_is_reported_not_raised(monkeypatch):
    def boom(R, steps):
        raise RuntimeError("device lost")
    _patch(monkeypatch, boom)
    out = bench.time_iteration_sweep({"name": "w", "params": {"iters": 4}}, None, None, 50)
    assert out["error"] == "RuntimeError: device lost"
