"""The MIP filter variants of Sec. 3.3 (the Sec. 4.4.2 ablation) on the GPU
vs the oracle, element by element: no filter, and the per-pixel Jacobian of
AA-2DGS; plus the box filter of the supersampled reference."""
import ctypes

import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_gpu_forward import _check_view, _renderer

pytestmark = pytest.mark.gpu

NONE, PIXEL = 1, 2


@pytest.mark.parametrize("seed,mode,sigma_f", [(1, NONE, 0.5), (2, PIXEL, 0.5), (3, PIXEL, 2.0), (4, PIXEL, 0.0)])
def test_forward_mip_variants_tiny(seed, mode, sigma_f):
    rng = np.random.default_rng(500 + seed)
    surf = _tiny.random_scene(rng, n=300, spread=0.5, scale=(0.01, 0.08))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=47)], "tiny")
    r = _renderer(sc, params=dict(sigma_f=sigma_f, mip_mode=mode, bg=(0.1, 0.2, 0.3)))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


@pytest.mark.parametrize("mode", [0, NONE, PIXEL])
def test_forward_checkerboard_plane(mode):
    """A 40k-surfel checkerboard plane receding towards the horizon at
    160 x 120 (the ablation's scene at a size the oracle renders whole):
    magnified surfels in front, minified and nearly edge-on ones far away."""
    sc = S.checkerboard_plane(n_side=200, spacing=0.1, cell=1.0, width=160, height=120)
    r = _renderer(sc, params=dict(mip_mode=mode))
    r.forward()
    assert r.read_status() == 0
    ref, gpu = _check_view(r, sc, 0)
    assert (gpu[:, 3] > 0.5).sum() > 5000


def test_per_pixel_filter_is_forward_only():
    import torch
    from paper_2605_05876_gb300 import _lib
    sc = S.sphere_4k(n=512, res=32)
    r = _renderer(sc, params=dict(mip_mode=PIXEL))
    r.forward()
    torch.cuda.synchronize()
    with pytest.raises(_lib.SS3DError):
        r.backward(torch.zeros(r.n_pixels, 4, device="cuda"))


def test_box_downsample_averages_blocks():
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import _ptr, _stream
    rng = np.random.default_rng(3)
    for (W, H, f) in [(64, 48, 2), (30, 20, 5), (16, 16, 1)]:
        img = rng.normal(size=(H, W, 4)).astype(np.float32)
        src = torch.from_numpy(img).cuda()
        out = torch.full((H // f, W // f, 4), np.nan, device="cuda")
        _lib.check(_lib.lib().ss_box_downsample(_ptr(src), W, H, f, _ptr(out), _stream()))
        torch.cuda.synchronize()
        # the same FP32 sums in the same order (rows of the block, then columns)
        acc = np.zeros((H // f, W // f, 4), np.float32)
        for j in range(f):
            for i in range(f):
                acc = (acc + img[j::f, i::f]).astype(np.float32)
        ref = (acc * np.float32(1.0 / (f * f))).astype(np.float32)
        assert np.array_equal(out.cpu().numpy(), ref)
    assert _lib.lib().ss_box_downsample(None, 4, 4, 2, None, None) == _lib.SS_ERR_INVALID_ARG
    assert _lib.lib().ss_box_downsample(_ptr(src), 15, 16, 2, _ptr(out), None) == _lib.SS_ERR_INVALID_ARG
