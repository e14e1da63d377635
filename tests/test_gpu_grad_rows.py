"""The per-record gradient rows cleared by the forward
(ss_render_params.zero_grad_in_forward): the Renderer skips the backward's
own clearing only for the first backward after its forward, in the same
graph capture or none (a backward needs its own forward in any case: it
turns the forward's layer state into its coefficients in place).  In the
deterministic mode each case gives bitwise the gradients of a backward that
clears its rows."""
import ctypes

import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")


class _Spy:
    """The library with ss_render_backward wrapped to record the flag each
    call receives."""

    def __init__(self, L):
        self.L = L
        self.flags = []

    def __getattr__(self, name):
        fn = getattr(self.L, name)
        if name != "ss_render_backward":
            return fn

        def call(*args):
            self.flags.append(int(args[2]._obj.zero_grad_in_forward))
            return fn(*args)
        return call


@pytest.fixture
def spy(monkeypatch):
    from paper_2605_05876_gb300 import _lib, api
    s = _Spy(_lib.lib())
    monkeypatch.setattr(api, "lib", lambda: s)
    return s


def _setup():
    import torch
    from paper_2605_05876_gb300.api import Renderer
    b = S.torus_sphere_100k(n=20000, res=96)
    r = Renderer(b, params=dict(deterministic=1))
    g = torch.Generator(device="cuda").manual_seed(11)
    d_rgba = torch.randn(r.rgba.shape, device="cuda", generator=g)
    d_aov = torch.randn(r.aov.shape, device="cuda", generator=g)
    return r, d_rgba, d_aov


def _grads(r):
    import torch
    torch.cuda.synchronize()
    assert r.read_status() == 0
    out = {k: r.grads[k].cpu().numpy().copy() for k in FIELDS}
    out["env"] = r.d_env.cpu().numpy().copy()
    return out


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


def test_rows_cleared_by_the_forward_give_the_clearing_backward(spy):
    r, d_rgba, d_aov = _setup()
    r.forward()
    r._rows_clear = None             # as if the forward's clearing were unknown
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    ref = _grads(r)
    r.forward()
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    _same(ref, _grads(r))
    assert spy.flags == [0, 1]


def test_graph_captures_pair_forward_and_backward(spy):
    """Forward and backward captured in one graph skip the backward's
    clearing; captured in two graphs (replayed in turn), the backward
    clears its rows in every replay."""
    import torch
    r, d_rgba, d_aov = _setup()
    r.forward()
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    ref = _grads(r)

    def capture(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            fn()
        return cg

    def bwd():
        r.zero_grads()
        r.backward(d_rgba, d_aov)

    def step():
        r.forward()
        bwd()

    spy.flags.clear()
    g = capture(step)                # eager warm-up step, then the captured step
    assert spy.flags == [1, 1]
    for _ in range(2):
        g.replay()
        _same(ref, _grads(r))
    del g

    spy.flags.clear()
    gf = capture(r.forward)
    gb = capture(bwd)                # the forward it follows was captured in another graph
    assert spy.flags == [0, 0]
    for _ in range(2):
        gf.replay()
        gb.replay()
        _same(ref, _grads(r))
    del gf, gb
    torch.cuda.synchronize()
    assert ctypes.sizeof(r.prm) == 128 and r.prm.zero_grad_in_forward == 0
