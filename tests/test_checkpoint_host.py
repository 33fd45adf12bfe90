"""Checkpoint / resume of Lloyd's iteration, on the host.

The moments and the update come from stand-ins for the GPU calls (a smooth
function of the points with a known gradient, and the update on the host), so what is tested is the loop around it: a
run interrupted by an exception and resumed from its checkpoint ends with
the same points as an uninterrupted run, resuming with no checkpoint written
starts from the given points, and no temporary file is left behind.
"""
import os

import pytest
import torch

from paper_2412_04514_gb300 import api


def fake_moments(q, params=None):
    # M2 = |q - 0.5|^2 / 2 per point and V = 1: each step moves p halfway to 0.5
    m2 = 0.5 * ((q.to(torch.float64) - 0.5) ** 2).sum(1)
    vol = torch.ones(q.shape[0], dtype=torch.float64)
    cen = torch.zeros(q.shape[0], 3, dtype=torch.float64)
    return vol, cen, m2


def fake_step(p, grad, vol, params=None):
    # the update the library's vt_lloyd_step applies, on the host
    return (p.to(torch.float64) - grad.to(torch.float64) / (2.0 * vol[:, None])).to(torch.float32)


@pytest.fixture(autouse=True)
def stand_in(monkeypatch):
    monkeypatch.setattr(api, "voronoi_moments", fake_moments)
    monkeypatch.setattr(api, "lloyd_step", fake_step)


def start_points():
    return torch.rand(50, 3, generator=torch.Generator().manual_seed(3))


def test_interrupted_run_resumes_to_the_same_points(tmp_path):
    p0 = start_points()
    full = api.lloyd(p0, 7)
    ck = str(tmp_path / "lloyd.pt")

    def stop_at_five(it, loss):
        if it == 4:
            raise KeyboardInterrupt

    with pytest.raises(KeyboardInterrupt):
        api.lloyd(p0, 7, checkpoint=ck, checkpoint_every=2, callback=stop_at_five)
    state = torch.load(ck, weights_only=True)
    assert state["iteration"] == 4  # saved after iterations 2 and 4; the fifth never finished
    resumed = api.lloyd(p0, 7, checkpoint=ck, checkpoint_every=2, resume=True)
    assert torch.equal(full, resumed)
    assert torch.load(ck, weights_only=True)["iteration"] == 7
    assert sorted(os.listdir(tmp_path)) == ["lloyd.pt"]


def test_resume_without_a_checkpoint_starts_from_the_points(tmp_path):
    p0 = start_points()
    ck = str(tmp_path / "none.pt")
    assert torch.equal(api.lloyd(p0, 3, checkpoint=ck, resume=True), api.lloyd(p0, 3))
    assert os.path.exists(ck)
