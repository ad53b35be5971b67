"""The CUDA flight-scene renderer (input generation for the streaming
workload) draws the host renderer's pixels: same scene tables, same pose,
same lens.  Small frames at poses on a straight leg and on a turn (camera
heading rotated)."""
import numpy as np
import pytest
import torch

from paper_1902_09733_b300 import build, synth
from paper_1902_09733_b300.scene import GpuScene

pytestmark = pytest.mark.gpu


def test_gpu_renderer_matches_the_host_renderer():
    assert torch.cuda.is_available()
    build.build_scene()
    W, H = 416, 234
    s = W / 2704.0
    cam = (1400.0 * s, 1400.0 * s, (W - 1) / 2.0, (H - 1) / 2.0, -0.25, 0.07)
    poses = synth.lawnmower_path(3, 1500)
    scene = synth.FlightScene(3, synth.lawnmower_extent(poses), n_buildings=80)
    gs = GpuScene(scene)
    for i in (0, 400, 700, 1200):          # leg, leg, turn (yaw != 0), return leg (yaw = pi)
        want = scene.render(poses[i], W, H, cam)
        got = gs.render(poses[i], cam, W, H).cpu().numpy()
        diff = np.abs(got.astype(int) - want.astype(int))
        assert (diff == 0).mean() >= 0.999, (i, (diff == 0).mean(), diff.max())
        assert (diff <= 1).mean() >= 0.9999, (i, (diff <= 1).mean())
