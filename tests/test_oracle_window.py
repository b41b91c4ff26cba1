"""Pin for the oracle's windowed transition ora_langevin_step_window.

The windowed step evaluates the x-update of Eq. 8 only at the pixels of a
window of the image, for images too large to step whole in FP64 (the 8192^2
precision workload). Its pin is the already-pinned whole-image transition:
on small images, every window (corners, edges, wrap-around rows and columns,
interior, the whole image) must equal the same pixels of ora_langevin_step
exactly, with the blur, the denoiser, the projection and the noise all on.
A window that reached too little of the denoiser's receptive field, used
local instead of global noise indices or wrapped the blur wrongly would
differ at some of these windows.
"""
import numpy as np
import pytest

import synth


def _problem(orc, ny, nx, h, net, seed, mask=None, noise=True):
    rng = np.random.default_rng(seed)
    y = rng.random((ny, nx))
    return orc.Problem(y, h, 0.05, 1.0, 0.05, 1e-3, 2e-4, 1000 + seed, net=net, noise=noise,
                       mask=mask), rng


WINDOWS = [(0, 0, 5, 7), (0, 44, 6, 8), (33, 0, 7, 6), (35, 45, 5, 7), (12, 20, 9, 11),
           (0, 0, 40, 52), (18, 3, 1, 1), (39, 51, 1, 1)]


@pytest.mark.parametrize("kind", ["motion", "gauss"])
def test_window_equals_whole_image_step(orc, kind):
    h = synth.motion_kernel(7, 0.7) if kind == "motion" else synth.gaussian_kernel(9, 1.8)
    dw = synth.denoiser_weights(4, 8, seed=5)
    net = orc.Net.from_weights(dw)
    p, rng = _problem(orc, 40, 52, h, net, 3)
    x = np.clip(p.y + 0.1 * rng.standard_normal(p.y.shape), -0.2, 1.2)
    for t in (0, 7):
        whole = orc.langevin_step(p, x, t, chain=2)
        for (i0, j0, wy, wx) in WINDOWS:
            win = orc.langevin_step_window(p, x, t, i0, j0, wy, wx, chain=2)
            np.testing.assert_array_equal(win, whole[i0:i0 + wy, j0:j0 + wx])


def test_window_without_denoiser_and_with_mask(orc):
    rng = np.random.default_rng(9)
    mask = (rng.random((40, 52)) < 0.4).astype(np.float64)
    for m, net in ((None, None), (mask, orc.Net.from_weights(synth.denoiser_weights(3, 8, 2)))):
        p, rng2 = _problem(orc, 40, 52, synth.uniform_kernel(5), net, 4, mask=m)
        x = rng2.random(p.y.shape)
        whole = orc.langevin_step(p, x, 11)
        for (i0, j0, wy, wx) in WINDOWS:
            win = orc.langevin_step_window(p, x, 11, i0, j0, wy, wx)
            np.testing.assert_array_equal(win, whole[i0:i0 + wy, j0:j0 + wx])


def test_window_rejects_bad_windows(orc):
    p, _ = _problem(orc, 20, 20, synth.uniform_kernel(3), None, 1)
    x = np.zeros((20, 20))
    for args in ((-1, 0, 2, 2), (0, 0, 21, 2), (19, 19, 2, 1), (0, 0, 0, 3)):
        with pytest.raises(ValueError):
            orc.langevin_step_window(p, x, 0, *args)
