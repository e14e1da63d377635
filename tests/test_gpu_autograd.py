"""The torch.autograd wrapper returns the library's gradients."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_autograd_matches_direct_backward():
    import torch
    from paper_2605_05876_gb300 import scenes as S
    from paper_2605_05876_gb300.api import SURFEL_FIELDS, Renderer, render
    sc = S.sphere_4k(n=1024, res=48)
    r = Renderer(sc)
    leaves = [r.params_t[k].requires_grad_(True) for k in SURFEL_FIELDS] + [r.env.requires_grad_(True)]
    rgba, aov = render(r, *leaves)
    g = torch.Generator(device="cuda").manual_seed(0)
    G = torch.randn(rgba.shape, device="cuda", generator=g)
    Ga = torch.randn(aov.shape, device="cuda", generator=g)
    ((rgba * G).sum() + (aov * Ga).sum()).backward()
    got = {k: t.grad.clone() for k, t in zip(SURFEL_FIELDS + ("env",), leaves)}
    # the same gradients through the direct calls
    r.zero_grads()
    r.forward()
    r.backward(G, Ga)
    # two runs differ only in the order of the atomic sums
    for k in SURFEL_FIELDS:
        assert (got[k] - r.grads[k]).norm() <= 1e-5 * r.grads[k].norm() + 1e-12, k
    assert (got["env"] - r.d_env).norm() <= 1e-5 * r.d_env.norm() + 1e-12
    assert any(got[k].abs().sum() > 0 for k in SURFEL_FIELDS)
