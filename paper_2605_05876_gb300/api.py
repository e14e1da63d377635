"""Device-resident front end over the C ABI.

``Renderer`` keeps one batch (surfels of one or more scenes, their views,
one environment map per scene) in HBM as torch tensors and calls the
library's entry points on torch's current CUDA stream.  PyTorch provides the
memory and the stream; all arithmetic runs in libss3d.so.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib as C
from ._lib import check, lib

SURFEL_FIELDS = ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_cameras(cams) -> ctypes.Array:
    arr = (C.ss_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].R[:] = [float(v) for v in np.asarray(c.R, np.float32).ravel()]
        arr[i].t[:] = [float(v) for v in np.asarray(c.t, np.float32).ravel()]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(np.float32(v)) for v in (c.fx, c.fy, c.cx, c.cy))
        arr[i].width, arr[i].height, arr[i].scene = int(c.width), int(c.height), int(c.scene)
    return arr


def default_params(**overrides) -> C.ss_render_params:
    p = C.ss_render_params()
    lib().ss_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "bg":
            p.bg[:] = list(v)
        else:
            setattr(p, k, v)
    return p


class Renderer:
    """One batch resident on the GPU.

    scene: ``paper_2605_05876_gb300.scenes.Scene`` (numpy inputs).
    params: overrides of ss_render_params fields (r_cut, sigma_f, ...).
    """

    def __init__(self, scene, params: dict | None = None, env_levels: int = 6, irr_size=(32, 16),
                 with_backward: bool = True, capacity_slack: float = 1.3, device: str = "cuda",
                 share_from: "Renderer | None" = None, screen_grad: bool = False):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.scene = scene
        s = scene.surfels
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(self.dev)
        if share_from is not None:   # same surfels and env maps, other views
            self.params_t = share_from.params_t
        else:
            self.params_t = {k: f32(getattr(s, k)) for k in SURFEL_FIELDS}
        self.n_surfels = s.n
        self.n_views = len(scene.cameras)
        self.n_scenes = scene.n_scenes
        self._cams_host = make_cameras(scene.cameras)
        self.cams_dev = torch.frombuffer(bytearray(bytes(self._cams_host)), dtype=torch.uint8).to(self.dev)
        self._offsets = (ctypes.c_int64 * (self.n_scenes + 1))(*[int(v) for v in scene.scene_offsets])
        self.desc = C.ss_batch_desc(self.n_scenes, self.n_views, self._offsets, self._cams_host,
                                    ctypes.c_void_p(self.cams_dev.data_ptr()))
        self.sizes = [(int(c.width), int(c.height)) for c in scene.cameras]
        self.pixel_offsets = np.concatenate([[0], np.cumsum([w * h for w, h in self.sizes])]).astype(np.int64)
        self.n_pixels = int(self.pixel_offsets[-1])
        # environment
        He, We, _ = scene.envs[0].shape
        self.ed = C.ss_env_desc(We, He, env_levels, irr_size[0], irr_size[1])
        ni, ns, na = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().ss_env_sizes(ctypes.byref(self.ed), ctypes.byref(ni), ctypes.byref(ns), ctypes.byref(na)),
              "ss_env_sizes")
        S = self.n_scenes
        self.prm = default_params(**(params or {}))
        self.prm.screen_grad = int(screen_grad)
        if share_from is not None:
            self.env, self.irr, self.spec, self.aux, self.lut = (share_from.env, share_from.irr, share_from.spec,
                                                                 share_from.aux, share_from.lut)
        else:
            self.env = torch.from_numpy(np.stack([np.asarray(e, np.float32) for e in scene.envs])).to(self.dev)
            self.irr = torch.zeros(S, ni.value, device=self.dev)
            self.spec = torch.zeros(S, ns.value, device=self.dev)
            self.aux = torch.zeros(S, na.value, device=self.dev)
            self.lut = torch.zeros(self.prm.lut_n, self.prm.lut_n, 2, device=self.dev)
            check(lib().ss_brdf_lut(_ptr(self.lut), self.prm.lut_n, _stream()), "ss_brdf_lut")
            self.prefilter_env()
        self.maps = C.ss_env_maps(_ptr(self.irr), _ptr(self.spec), _ptr(self.lut))
        # outputs
        self.rgba = torch.zeros(self.n_pixels, 4, device=self.dev)
        # AOV planes: albedo 3, roughness, metallic, normal 3, depth; with the
        # depth-consolidation term (params cons=1) a tenth plane holds it
        self.aov = torch.zeros(C.SS_N_AOV + int(self.prm.cons), self.n_pixels, device=self.dev)
        self.with_backward = with_backward
        self.capacity_slack = capacity_slack
        self.ws = None
        self.plan_capacity()

    # -- surfel parameters as the ABI struct
    def surfels_struct(self) -> C.ss_surfels:
        p = self.params_t
        return C.ss_surfels(*(ctypes.c_void_p(p[k].data_ptr()) for k in SURFEL_FIELDS))

    def prefilter_env(self):
        check(lib().ss_env_prefilter(ctypes.byref(self.ed), self.n_scenes, _ptr(self.env), _ptr(self.irr),
                                     _ptr(self.spec), _ptr(self.aux), _stream()), "ss_env_prefilter")

    def plan_capacity(self, max_instances: int | None = None):
        torch = self.torch
        if max_instances is None:
            probe = default_params()
            ctypes.memmove(ctypes.byref(probe), ctypes.byref(self.prm), ctypes.sizeof(probe))
            probe.max_instances = 1
            nb = ctypes.c_size_t()
            check(lib().ss_workspace_size(ctypes.byref(self.desc), ctypes.byref(probe), ctypes.byref(self.ed), 0,
                                          ctypes.byref(nb)),
                  "ss_workspace_size")
            ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.dev)
            cnt = ctypes.c_int64()
            check(lib().ss_count_instances(ctypes.byref(self.desc), ctypes.byref(self.surfels_struct()),
                                           ctypes.byref(self.prm), ctypes.byref(self.ed), ctypes.byref(self.maps),
                                           _ptr(ws), nb.value, ctypes.byref(cnt), _stream()), "ss_count_instances")
            self.counted_instances = int(cnt.value)
            max_instances = int(math.ceil(cnt.value * self.capacity_slack)) + 4096
            del ws
        self.prm.max_instances = max_instances
        nb = ctypes.c_size_t()
        check(lib().ss_workspace_size(ctypes.byref(self.desc), ctypes.byref(self.prm), ctypes.byref(self.ed),
                                      int(self.with_backward), ctypes.byref(nb)), "ss_workspace_size")
        self.ws_bytes = nb.value
        self.ws = torch.empty(nb.value, dtype=torch.uint8, device=self.dev)
        self._rows_clear = None   # a new workspace: its gradient rows hold nothing yet

    def _capture_id(self) -> int:
        cid = ctypes.c_uint64()
        check(lib().ss_stream_capture_id(_stream(), ctypes.byref(cid)), "ss_stream_capture_id")
        return int(cid.value)

    def forward(self):
        # with backward state, the forward also clears the per-record gradient
        # rows (params zero_grad_in_forward); the first backward after it, in
        # the same graph capture or none, then skips that clearing
        self._rows_clear = None
        self.prm.zero_grad_in_forward = int(self.with_backward)
        try:
            check(lib().ss_render_forward(ctypes.byref(self.desc), ctypes.byref(self.surfels_struct()),
                                          ctypes.byref(self.prm), ctypes.byref(self.ed), ctypes.byref(self.maps),
                                          _ptr(self.rgba), _ptr(self.aov), _ptr(self.ws), self.ws_bytes, _stream()),
                  "ss_render_forward")
        finally:
            self.prm.zero_grad_in_forward = 0
        if self.with_backward:
            self._rows_clear = self._capture_id()
        return self.rgba, self.aov

    def zero_grads(self, share_from: "Renderer | None" = None):
        torch = self.torch
        if share_from is not None:
            self.grads, self.d_irr, self.d_spec, self.d_env = (share_from.grads, share_from.d_irr,
                                                               share_from.d_spec, share_from.d_env)
            return
        if hasattr(self, "grads"):
            for v in self.grads.values():
                v.zero_()
            self.d_irr.zero_()
            self.d_spec.zero_()
            self.d_env.zero_()
            if self.prm.screen_grad:
                self.screen_grad_norm.zero_()
                self.screen_grad_views.zero_()
            return
        self.grads = {k: torch.zeros_like(v) for k, v in self.params_t.items()}
        self.d_irr = torch.zeros_like(self.irr)
        self.d_spec = torch.zeros_like(self.spec)
        self.d_env = torch.zeros_like(self.env)
        if self.prm.screen_grad:
            # densification statistic (Sec. 3.6.1, Eq. ss_grad): per surfel the summed
            # |(g_x, g_y)| of its fragments and the number of views it appeared in
            self.screen_grad_norm = torch.zeros(self.n_surfels, device=self.dev)
            self.screen_grad_views = torch.zeros(self.n_surfels, device=self.dev)

    def env_backward(self):
        # with params deterministic=1 the level terms are added in a fixed order
        name = "ss_env_prefilter_backward_ordered" if self.prm.deterministic else "ss_env_prefilter_backward"
        check(getattr(lib(), name)(ctypes.byref(self.ed), self.n_scenes, _ptr(self.d_irr), _ptr(self.d_spec),
                                   _ptr(self.aux), _ptr(self.d_env), _stream()), name)

    def stats(self):
        st = C.ss_stats()
        check(lib().ss_read_stats(_ptr(self.ws), ctypes.byref(st), _stream()), "ss_read_stats")
        return {k: int(getattr(st, k)) for k, _ in C.ss_stats._fields_ if k != "reserved"}

    def backward(self, d_rgba, d_aov=None, env_grad: bool = True):
        """Accumulate gradients of sum(d_rgba * rgba) + sum(d_aov * aov) into
        self.grads (surfel params) and self.d_env (base env texels).  One
        backward per forward: it consumes the forward's layer state."""
        if not hasattr(self, "grads"):
            self.zero_grads()
        ssg = (_ptr(self.screen_grad_norm), _ptr(self.screen_grad_views)) if self.prm.screen_grad else (None, None)
        g = C.ss_surfel_grads(*(ctypes.c_void_p(self.grads[k].data_ptr()) for k in SURFEL_FIELDS), *ssg)
        ge = C.ss_env_map_grads(_ptr(self.d_irr), _ptr(self.d_spec))
        rows_clear = self._rows_clear is not None and self._rows_clear == self._capture_id()
        self._rows_clear = None
        self.prm.zero_grad_in_forward = int(rows_clear)
        try:
            check(lib().ss_render_backward(ctypes.byref(self.desc), ctypes.byref(self.surfels_struct()),
                                           ctypes.byref(self.prm), ctypes.byref(self.ed), ctypes.byref(self.maps),
                                           _ptr(self.rgba), _ptr(self.aov), _ptr(d_rgba.contiguous()),
                                           _ptr(d_aov.contiguous() if d_aov is not None else None), ctypes.byref(g),
                                           ctypes.byref(ge), _ptr(self.ws), self.ws_bytes, _stream()),
                  "ss_render_backward")
        finally:
            self.prm.zero_grad_in_forward = 0
        if env_grad:
            self.env_backward()
        return self.grads


    # screen tiles made of 8 x 4 warp blocks (at most 8 per tile), forward
    # staging depth, launch shapes; searched in this order
    TUNE_SPACE = {"tile": ((16, 16), (16, 8), (32, 8), (8, 16), (8, 8)), "stage_depth": (1, 2, 3),
                  "fwd_warps": (1, 2, 4), "bwd_warps": (2, 4, 8), "pbwd_block": (64, 128, 256)}

    def state_dict(self) -> dict:
        """The surfel parameters the renderer reads and the base env map
        (copies), for torch.save: with Adam.state_dict, a checkpoint of the
        inverse-rendering loop."""
        return {"params": {k: v.detach().clone() for k, v in self.params_t.items()}, "env": self.env.detach().clone()}

    def load_state_dict(self, st: dict):
        """Restore a state_dict into this renderer's tensors (same surfel
        count and env shape); the prefiltered maps are recomputed by the next
        prefilter_env."""
        for k, v in self.params_t.items():
            v.copy_(st["params"][k])
        self.env.copy_(st["env"])

    def compact_workspace(self, dense: int = 2, slack: float = 1.25):
        """Size the workspace by this batch's work instead of its bounds: the
        rasterisers' block lists by the candidates a forward counts
        (ss_stats.candidates; the first forward runs with no room, which the
        binning counts all the same), then `dense` layers per pixel in planes
        of every pixel and the deeper ones in a pool sized by the (pixel,
        layer) pairs past `dense` that a second forward counts
        (ss_stats.pool_layers); each with `slack`.  Returns (candidates
        capacity, pool slots, workspace bytes)."""
        self.prm.dense_layers, self.prm.layer_pool, self.prm.max_candidates = int(dense), 0, 1
        self.plan_capacity(self.prm.max_instances)
        self.forward()
        self.prm.max_candidates = int(math.ceil(self.stats()["candidates"] * slack)) + 4096
        self.plan_capacity(self.prm.max_instances)
        self.forward()
        self.prm.layer_pool = int(math.ceil(self.stats()["pool_layers"] * slack)) + 1024
        self.plan_capacity(self.prm.max_instances)
        return self.prm.max_candidates, self.prm.layer_pool, self.ws_bytes

    def set_tile(self, tile):
        """Change the screen tile (width, height); the instance capacity and
        the workspace are planned again for it."""
        self.prm.tile_w, self.prm.tile_h = int(tile[0]), int(tile[1])
        self.ws = None
        self.plan_capacity()

    def autotune(self, d_rgba, d_aov=None, reps: int = 3, space: dict | None = None) -> dict:
        """Choose the tile shape, the forward staging depth and the launch
        shapes of ss_render_params that render and differentiate this batch
        fastest, one knob at a time in the order given, each candidate timed
        with CUDA events over `reps` forward+backward passes after one
        untimed pass.  These knobs change speed only, never results.
        Returns {knob: (chosen value, {value: ms per pass})}."""
        torch = self.torch
        space = space or self.TUNE_SPACE

        def one():
            self.forward()
            self.zero_grads()
            self.backward(d_rgba, d_aov, env_grad=False)

        def timed() -> float:
            one()
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                one()
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        chosen = {}
        for knob, values in space.items():
            times = {}
            for v in values:
                if knob == "tile":
                    self.set_tile(v)
                    key = f"{v[0]}x{v[1]}"
                else:
                    setattr(self.prm, knob, int(v))
                    key = int(v)
                times[key] = timed()
            best = min(times, key=times.get)
            if knob == "tile":
                w, h = (int(x) for x in best.split("x"))
                self.set_tile((w, h))
            else:
                setattr(self.prm, knob, best)
            chosen[knob] = (best, times)
        return chosen

    # -- adaptive density control (Sec. 3.6.2)
    def density_params(self, **overrides) -> C.ss_density_params:
        """ss_density_params with the library's defaults, the grid cell set
        from this batch's surfel scales (twice the median of max(s_u, s_v)
        over a sample) unless given, and the given overrides."""
        p = C.ss_density_params()
        lib().ss_default_density(ctypes.byref(p))
        if "cell" not in overrides:
            ls = self.params_t["log_scale"]
            step = max(1, self.n_surfels // 65536)
            sample = ls[::step].max(dim=1).values.float().cpu().numpy()
            overrides["cell"] = float(2.0 * np.exp(np.median(sample))) if sample.size else 1.0
        for k, v in overrides.items():
            setattr(p, k, v)
        return p

    def _density_ws(self, n: int):
        nb = ctypes.c_size_t()
        check(lib().ss_density_workspace_size(int(n), ctypes.byref(nb)), "ss_density_workspace_size")
        if getattr(self, "_dws", None) is None or self._dws.numel() < nb.value:
            self._dws = self.torch.empty(max(nb.value, 1), dtype=self.torch.uint8, device=self.dev)
        return self._dws, nb.value

    def density_neighbours(self, dp: C.ss_density_params):
        """(mean_dist, nn_dist, flags) device tensors of ss_density_neighbours."""
        torch = self.torch
        n = self.n_surfels
        mean = torch.empty(n, device=self.dev)
        nn = torch.empty(n, device=self.dev)
        flags = torch.empty(n, dtype=torch.int32, device=self.dev)
        ws, nb = self._density_ws(n)
        check(lib().ss_density_neighbours(ctypes.byref(self.surfels_struct()), self._offsets, self.n_scenes,
                                          ctypes.byref(dp), _ptr(mean), _ptr(nn), _ptr(flags), _ptr(ws), nb,
                                          _stream()), "ss_density_neighbours")
        return mean, nn, flags

    def density_plan(self, dp: C.ss_density_params, mean, nn, flags, g_norm=None, g_views=None):
        """(action int32 [N], out_offset int64 [N+1]) of ss_density_plan, by
        default from the accumulated screen-space statistic."""
        torch = self.torch
        n = self.n_surfels
        g_norm = self.screen_grad_norm if g_norm is None else g_norm
        g_views = self.screen_grad_views if g_views is None else g_views
        action = torch.empty(n, dtype=torch.int32, device=self.dev)
        off = torch.empty(n + 1, dtype=torch.int64, device=self.dev)
        ws, nb = self._density_ws(n)
        check(lib().ss_density_plan(_ptr(self.params_t["log_scale"]), _ptr(g_norm), _ptr(g_views), _ptr(mean),
                                    _ptr(nn), _ptr(flags), n, ctypes.byref(dp), _ptr(action), _ptr(off), _ptr(ws),
                                    nb, _stream()), "ss_density_plan")
        return action, off

    def densify(self, dp: C.ss_density_params | None = None, adam: "Adam | None" = None) -> dict:
        """One pass of adaptive density control over the batch: neighbour
        statistics, the split / prune plan from the screen-space statistic
        accumulated since the last zero_grads (screen_grad=True), and the new
        surfel arrays.  The renderer is re-planned for the new count and its
        gradients and statistic are zeroed.  With `adam`, its surfel groups
        follow: raw values of kept and split surfels are carried over,
        moments of children start at zero.  Returns the counts."""
        torch = self.torch
        if not self.prm.screen_grad:
            raise ValueError("density control reads the screen-space statistic: Renderer(screen_grad=True)")
        dp = dp or self.density_params()
        n = self.n_surfels
        mean, nn, flags = self.density_neighbours(dp)
        action, off = self.density_plan(dp, mean, nn, flags)
        bounds = off[torch.tensor([int(v) for v in self._offsets], device=self.dev)].cpu().tolist()
        n_new = int(bounds[-1])
        new = {k: torch.empty((n_new,) + tuple(v.shape[1:]), device=self.dev) for k, v in self.params_t.items()}
        sin, sout = self.surfels_struct(), C.ss_surfels(*(_ptr(new[k]) for k in SURFEL_FIELDS))
        check(lib().ss_density_apply(ctypes.byref(sin), n, _ptr(action), _ptr(off), float(dp.split_scale),
                                     ctypes.byref(sout), _stream()), "ss_density_apply")
        counts = torch.bincount(action.long(), minlength=3).cpu().tolist()
        old = self.params_t
        self.params_t = new
        self.n_surfels = n_new
        self._offsets = (ctypes.c_int64 * (self.n_scenes + 1))(*bounds)
        self.desc.scene_offsets_host = self._offsets
        if hasattr(self, "grads"):
            del self.grads
        self.zero_grads()
        self.ws = None
        self.plan_capacity()
        if adam is not None:
            groups, moments = {}, {}
            for k, (raw, grad, act, lr, activation) in adam.groups.items():
                if k not in SURFEL_FIELDS:
                    groups[k], moments[k] = (raw, grad, act, lr, activation), adam.moments[k]
                    continue
                if raw.data_ptr() == old[k].data_ptr():
                    nraw = new[k]
                else:
                    nraw = self.compact_rows(raw, action, off, n_new, zero_children=False)
                m, v = adam.moments[k]
                moments[k] = (self.compact_rows(m, action, off, n_new, zero_children=True),
                              self.compact_rows(v, action, off, n_new, zero_children=True))
                groups[k] = (nraw, self.grads[k], None if act is None else new[k], lr, activation)
            adam.replace(groups, moments)
        return {"before": n, "after": n_new, "pruned": counts[0], "kept": counts[1], "split": counts[2]}

    def compact_rows(self, t, action, off, n_new: int, zero_children: bool):
        """ss_density_compact of a per-surfel tensor [N, ...] into a new one."""
        n = action.numel()
        width = t.numel() // max(n, 1)
        out = self.torch.empty((n_new,) + tuple(t.shape[1:]), device=self.dev)
        check(lib().ss_density_compact(_ptr(t.contiguous()), width, n, _ptr(action), _ptr(off), int(zero_children),
                                       _ptr(out), _stream()), "ss_density_compact")
        return out

    def read_status(self) -> int:
        return int(lib().ss_read_status(_ptr(self.ws), _stream()))

    def set_cameras(self, cams):
        """Replace the views' poses/intrinsics (same sizes and scenes)."""
        arr = make_cameras(cams)
        for i, c in enumerate(cams):
            if (c.width, c.height, c.scene) != (self._cams_host[i].width, self._cams_host[i].height,
                                                 self._cams_host[i].scene):
                raise ValueError("set_cameras keeps sizes and scenes")
        src = self.torch.frombuffer(bytearray(bytes(arr)), dtype=self.torch.uint8)
        self.cams_dev.copy_(src, non_blocking=False)
        ctypes.memmove(self._cams_host, arr, ctypes.sizeof(arr))

    # -- views of the outputs
    def view_slice(self, v: int) -> slice:
        return slice(int(self.pixel_offsets[v]), int(self.pixel_offsets[v + 1]))

    def view_rgba(self, v: int):
        w, h = self.sizes[v]
        return self.rgba[self.view_slice(v)].reshape(h, w, 4)

    def view_aov(self, v: int):
        w, h = self.sizes[v]
        return self.aov[:, self.view_slice(v)].reshape(self.aov.shape[0], h, w)


def profile_begin():
    check(lib().ss_profile_begin(), "ss_profile_begin")


def profile_end() -> dict:
    t = C.ss_stage_times()
    check(lib().ss_profile_end(ctypes.byref(t)), "ss_profile_end")
    return {name: (float(t.ms[i]), int(t.launches[i])) for i, name in enumerate(C.STAGES)}


def launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    n = ctypes.c_int64()
    check(lib().ss_launch_count(ctypes.byref(n)), "ss_launch_count")
    return int(n.value)


# ------------------------------------------------------------------------
# optimisation

SURFEL_ACTIVATIONS = {"pos": C.SS_ACT_IDENTITY, "quat": C.SS_ACT_IDENTITY, "log_scale": C.SS_ACT_IDENTITY,
                      "albedo": C.SS_ACT_SIGMOID, "roughness": C.SS_ACT_SIGMOID, "metallic": C.SS_ACT_SIGMOID}


class Adam:
    """Fused Adam (ss_adam_step) over named parameter groups.

    Each group is (raw, grad, act, lr, activation): raw values owned by the
    optimiser, the gradient w.r.t. the activated values the renderer reads
    (act; may be raw itself for identity activations) and its learning rate.
    """

    def __init__(self, groups: dict, beta1=0.9, beta2=0.999, eps=1e-8):
        import torch
        if not 1 <= len(groups) <= C.SS_MAX_ADAM_GROUPS:
            raise ValueError("1 .. 16 groups")
        self.p = C.ss_adam_params()
        lib().ss_default_adam(ctypes.byref(self.p))
        self.p.beta1, self.p.beta2, self.p.eps = beta1, beta2, eps
        self.t = 0
        self.replace(groups, {k: (torch.zeros_like(g[0]), torch.zeros_like(g[0])) for k, g in groups.items()})

    def replace(self, groups: dict, moments: dict):
        """Point the optimiser at new tensors (same group names), e.g. after
        density control changed the surfel count; the step count is kept."""
        import torch
        self.groups = groups
        self.moments = moments
        arr = (C.ss_adam_group * len(groups))()
        for i, (k, (raw, grad, act, lr, activation)) in enumerate(groups.items()):
            m, v = self.moments[k]
            for t in (raw, grad, m, v) + ((act,) if act is not None else ()):
                if not t.is_contiguous() or t.dtype != torch.float32:
                    raise ValueError(f"group {k}: float32 contiguous tensors")
            arr[i] = C.ss_adam_group(_ptr(raw), _ptr(grad), _ptr(m), _ptr(v),
                                     _ptr(act) if act is not None and act.data_ptr() != raw.data_ptr() else None,
                                     raw.numel(), float(lr), int(activation))
        self._arr = arr

    def step(self):
        self.t += 1
        self.p.step = self.t
        check(lib().ss_adam_step(self._arr, len(self.groups), ctypes.byref(self.p), _stream()), "ss_adam_step")

    def state_dict(self) -> dict:
        """Step count, raw values and moments of every group (copies), for
        torch.save; the activated copies belong to the renderer's state."""
        return {"t": self.t,
                "raw": {k: g[0].detach().clone() for k, g in self.groups.items()},
                "m": {k: m.detach().clone() for k, (m, _) in self.moments.items()},
                "v": {k: v.detach().clone() for k, (_, v) in self.moments.items()}}

    def load_state_dict(self, st: dict):
        """Restore a state_dict into this optimiser's tensors (same groups and sizes)."""
        self.t = int(st["t"])
        for k, g in self.groups.items():
            g[0].copy_(st["raw"][k])
            self.moments[k][0].copy_(st["m"][k])
            self.moments[k][1].copy_(st["v"][k])


def loss_sil_iou(rgba, mask, view_offsets, d_rgba, loss, scale: float = 1.0):
    """Silhouette soft-IoU loss (Eq. sil_loss) per view on the coverage
    channel of rgba [P,4] against mask [P]; view_offsets: int64 device tensor
    [V+1]; loss [V] written, its gradient added into d_rgba[:, 3]."""
    check(lib().ss_loss_sil_iou(_ptr(rgba), _ptr(mask), _ptr(view_offsets), int(view_offsets.numel() - 1),
                                float(scale), _ptr(d_rgba), _ptr(loss), _stream()), "ss_loss_sil_iou")


def loss_l1(out, target, d_out, loss, scale: float = 1.0):
    """loss[0] = scale * sum|out - target|, d_out = scale * sign(out - target) (device tensors)."""
    check(lib().ss_loss_l1(_ptr(out), _ptr(target), out.numel(), float(scale), _ptr(d_out), _ptr(loss), _stream()),
          "ss_loss_l1")


# ------------------------------------------------------------------------
# autograd

class RenderFunction:
    """``torch.autograd.Function`` over a Renderer: forward renders RGBA and
    AOVs from the renderer's surfel parameters and environment map; backward
    calls ss_render_backward and ss_env_prefilter_backward and returns the
    gradients of the surfel parameters and of the base env map.

        rgba, aov = render(renderer, pos, quat, log_scale, albedo, roughness, metallic, env)

    The tensors passed in must be the renderer's own parameter tensors (the
    library reads them by pointer); their .grad receives the gradients."""

    @staticmethod
    def build():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, r, *tensors):
                for k, t in zip(SURFEL_FIELDS + ("env",), tensors):
                    own = r.env if k == "env" else r.params_t[k]
                    if t.data_ptr() != own.data_ptr():
                        raise ValueError(f"{k}: pass the renderer's own tensor")
                r.prefilter_env()
                rgba, aov = r.forward()
                ctx.r = r
                return rgba.clone(), aov.clone()

            @staticmethod
            def backward(ctx, d_rgba, d_aov):
                r = ctx.r
                r.zero_grads()
                r.backward(d_rgba.contiguous(), d_aov.contiguous() if d_aov is not None else None)
                return (None,) + tuple(r.grads[k].clone() for k in SURFEL_FIELDS) + (r.d_env.clone(),)

        return _F


_RENDER_FN = None


def render(r: "Renderer", *tensors):
    """Differentiable render (see RenderFunction)."""
    global _RENDER_FN
    if _RENDER_FN is None:
        _RENDER_FN = RenderFunction.build()
    return _RENDER_FN.apply(r, *tensors)
