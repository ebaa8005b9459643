"""The colour-histogram transformer (Sec. 4.1) on the GPU against the oracle, bit for bit.

Covers the hand-derived fixture, frames whose width makes every box row start at a
different byte phase and alignment, one-pixel and whole-frame boxes, boxes that end
at the last byte of the frame buffer, every bin layout up to d = 1024, the full
64-frame 1080p detector workload, and the rejections.
"""

import numpy as np
import pytest

import oracle
from oracle_pins import read_hist_golden
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import torch
    from paper_1812_07607_gb300 import build as B, dl as D
    assert torch.cuda.is_available()
    B.build()
    D.load()
    return D


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def _gpu_hist(dl, frames, boxes, bins):
    import torch
    return dl.color_hist(torch.from_numpy(frames).cuda(), torch.from_numpy(boxes).cuda(), bins).cpu().numpy()


def test_golden_fixture(dl, orc):
    frames, boxes, cases = read_hist_golden()
    for bins, counts in cases:
        got = _gpu_hist(dl, frames, boxes, bins)
        assert np.array_equal(got, orc.color_hist(frames, boxes, bins))
        for b, cnt in counts.items():
            x0, y0, x1, y1 = boxes[b, 1:]
            assert np.array_equal(got[b], np.array(cnt, np.float32) / np.float32((x1 - x0) * (y1 - y0)))


def _random_boxes(g, nF, H, Wd, n):
    boxes = []
    for _ in range(n):
        f = int(g.integers(0, nF))
        kind = g.integers(0, 4)
        if kind == 0:      # one pixel
            x0, y0 = int(g.integers(0, Wd)), int(g.integers(0, H))
            boxes.append([f, x0, y0, x0 + 1, y0 + 1])
        elif kind == 1:    # whole frame
            boxes.append([f, 0, 0, Wd, H])
        else:
            x0, y0 = int(g.integers(0, Wd)), int(g.integers(0, H))
            boxes.append([f, x0, y0, int(g.integers(x0 + 1, Wd + 1)), int(g.integers(y0 + 1, H + 1))])
    # the last pixel(s) of the buffer
    boxes += [[nF - 1, Wd - 1, H - 1, Wd, H], [nF - 1, 0, H - 1, Wd, H], [nF - 1, Wd - 7 if Wd > 7 else 0, H - 3 if H > 3 else 0, Wd, H]]
    return np.array(boxes, dtype=np.int32)


@pytest.mark.parametrize("shape", [(3, 23, 37), (2, 17, 1), (2, 5, 203), (1, 64, 64), (4, 9, 515)])
@pytest.mark.parametrize("bins", [(1, 1, 1), (8, 4, 4), (4, 3, 2), (16, 8, 8), (256, 1, 4), (5, 7, 3)])
def test_random_frames_equal_oracle(dl, orc, shape, bins):
    g = W.rng(7000 + shape[2] * 7 + bins[0])
    nF, H, Wd = shape
    frames = g.integers(0, 256, size=(nF, H, Wd, 3), dtype=np.uint8)
    # flat regions too: long runs of one bin
    frames[:, : H // 2, : Wd // 2] = g.integers(0, 256, size=3, dtype=np.uint8)
    boxes = _random_boxes(g, nF, H, Wd, 80)
    assert np.array_equal(_gpu_hist(dl, frames, boxes, bins), orc.color_hist(frames, boxes, bins))


def test_full_detector_workload(dl, orc):
    wl = W.traffic_boxes_1080p()
    got = _gpu_hist(dl, wl.frames, wl.boxes, wl.bins)
    assert np.array_equal(got, orc.color_hist(wl.frames, wl.boxes, wl.bins))


def test_rejections_and_empty(dl):
    import torch
    frames = torch.zeros((2, 8, 8, 3), dtype=torch.uint8, device="cuda")
    ok = torch.tensor([[0, 0, 0, 8, 8]], dtype=torch.int32, device="cuda")
    for bad in ([2, 0, 0, 1, 1], [0, 3, 0, 3, 1], [0, 0, 0, 9, 1], [0, -1, 0, 1, 1], [0, 0, 5, 1, 4]):
        with pytest.raises(dl.DLError) as ei:
            dl.color_hist(frames, torch.tensor([bad], dtype=torch.int32, device="cuda"), (4, 4, 4))
        assert ei.value.status == dl.DL_EINVAL
    for bins in ((0, 1, 1), (257, 1, 1), (16, 16, 8)):
        with pytest.raises(dl.DLError) as ei:
            dl.color_hist(frames, ok, bins)
        assert ei.value.status == dl.DL_EINVAL
    raw = torch.zeros(2 * 8 * 8 * 3 + 16, dtype=torch.uint8, device="cuda")
    misaligned = raw[1:1 + 2 * 8 * 8 * 3].view(2, 8, 8, 3)
    with pytest.raises(dl.DLError) as ei:
        dl.color_hist(misaligned, ok, (4, 4, 4))
    assert ei.value.status == dl.DL_EINVAL
    out = dl.color_hist(frames, torch.empty((0, 5), dtype=torch.int32, device="cuda"), (4, 4, 4))
    assert out.shape == (0, 64)
    h = dl.color_hist(frames, ok, (4, 4, 4)).cpu().numpy()
    assert h[0, 0] == 1.0 and h[0, 1:].sum() == 0.0
