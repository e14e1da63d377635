"""The C ABI library builds, loads and exports every entry point that
include/ss3d.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

from paper_2605_05876_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ss3d.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ss_status|void|const char\*)\s+(ss_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ss_render_forward", "ss_render_backward", "ss_env_prefilter", "ss_env_prefilter_backward",
              "ss_brdf_lut", "ss_workspace_size", "ss_read_status"):
        assert n in names


def test_library_exports_every_declared_symbol():
    build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) == set(declared_functions())


def test_struct_sizes_match_header():
    assert ctypes.sizeof(_lib.ss_camera) == 80
    assert ctypes.sizeof(_lib.ss_render_params) == 128
    assert ctypes.sizeof(_lib.ss_surfel_grads) == 64
    assert ctypes.sizeof(_lib.ss_stats) == 88


def test_struct_layouts_match_the_header_field_by_field():
    """Every struct the binding mirrors has the header's size and, field by
    field, the header's names and offsets: a C program generated from the
    ctypes definitions prints sizeof and offsetof of each (gcc, the plain C
    view of include/ss3d.h), so a field renamed, reordered or retyped on
    either side fails here."""
    import subprocess
    structs = [v for v in vars(_lib).values()
               if isinstance(v, type) and issubclass(v, ctypes.Structure) and hasattr(v, "_fields_")]
    assert len(structs) >= 12
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ss3d.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'    printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f in st._fields_:
            lines.append(f'    printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["    return 0;", "}"]
    out_dir = os.path.join(ROOT, "_build", "abi_layout")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "layout.c"), os.path.join(out_dir, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", exe, src])
    got = {}
    for line in subprocess.check_output([exe], text=True).splitlines():
        n, f, v = line.split()
        got[(n, f)] = int(v)
    for st in structs:
        n = st.__name__
        assert got[(n, "sizeof")] == ctypes.sizeof(st), n
        for f in st._fields_:
            assert got[(n, f[0])] == getattr(st, f[0]).offset, (n, f[0])


def _c_kind(decl: str) -> str:
    """Kind of a C parameter declaration: ptr, i32, i64, u32 or u64 (size_t
    is 64-bit unsigned on every target here), f32, f64."""
    decl = " ".join(decl.split())
    if "*" in decl:
        return "ptr"
    words = decl.replace("const ", "").split()
    t = words[0]
    return {"int32_t": "i32", "int": "i32", "ss_status": "i32", "int64_t": "i64", "uint32_t": "u32",
            "uint64_t": "u64", "size_t": "u64", "float": "f32", "double": "f64"}[t]


def _ctypes_kind(a) -> str:
    if a in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(a, type) and issubclass(a, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_uint32: "u32", ctypes.c_uint64: "u64",
            ctypes.c_float: "f32", ctypes.c_double: "f64"}[a]


def test_binding_signatures_match_the_header():
    """Each declared function's parameters, in order, have the kinds of the
    binding's argtypes (pointer, 32/64-bit integer, float), and its return
    type the binding's restype: an int32 passed for an int64 or a swapped
    pair of arguments fails here."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = re.findall(r"^\s*(ss_status|void|const char\*)\s+(ss_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.M | re.S)
    assert {n for _, n, _ in protos} == set(_lib.EXPORTS)
    for ret, name, args in protos:
        args = args.strip()
        want = [] if args in ("", "void") else [_c_kind(x) for x in args.split(",")]
        restype, argtypes = _lib.EXPORTS[name]
        assert [_ctypes_kind(t) for t in argtypes] == want, name
        assert restype == {"ss_status": ctypes.c_int32, "void": None, "const char*": ctypes.c_char_p}[ret], name


def test_constants_match_the_header():
    """Every integer #define SS_* of the header is a constant of the binding
    with the same value, and the binding has no SS_* constant the header
    lacks."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    lits = re.findall(r"^#define (SS_[A-Z0-9_]+) ([^\n]+)$", src, flags=re.M)
    # C integer literals: drop the suffixes (1ll, 0xfffffffell, 8u)
    defs = {n: eval(re.sub(r"(?<=[0-9a-fA-F])(?:ull|ULL|ll|LL|u|U|l|L)\b", "", v.strip())) for n, v in lits}
    ours = {n: v for n, v in vars(_lib).items() if n.startswith("SS_") and isinstance(v, int)}
    assert len(defs) >= 30
    assert defs == ours


def test_batch_limits_are_checked_on_the_host():
    """Record indices are 32-bit (SS_MAX_RECORDS) and (tile, block) items are
    numbered in 32 bits (SS_MAX_TILES): a batch past either is refused by the
    workspace query, one at the limit is planned."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    nb = ctypes.c_size_t()

    def query(n_views, n_surfels, w=16, h=16, tile=(8, 4)):
        p.tile_w, p.tile_h = tile
        cams = (_lib.ss_camera * n_views)()
        for c in cams:
            c.width, c.height, c.fx, c.fy = w, h, 10.0, 10.0
        off = (ctypes.c_int64 * 2)(0, n_surfels)
        d = _lib.ss_batch_desc(1, n_views, off, cams, None)
        return lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 0, ctypes.byref(nb))

    # records: views x the scene's surfels
    assert query(255, 1 << 24) == 0                              # 4.28e9 records
    assert query(256, 1 << 24) == _lib.SS_ERR_INVALID_ARG         # 2^32 records
    assert query(2, _lib.SS_MAX_RECORDS // 2) == 0                # exactly SS_MAX_RECORDS
    assert query(3, 0x55555555) == _lib.SS_ERR_INVALID_ARG        # 0xffffffff, scenes within their limit
    assert query(3, 0x55555554) == 0
    # tiles: 8 x 4 tiles of a 32768^2 view = 2^25 each
    assert query(4, 10, 32768, 32768) == 0                        # 2^27 tiles
    assert query(5, 10, 32768, 32768) == _lib.SS_ERR_INVALID_ARG


def test_host_side_argument_errors():
    """Host-detectable errors return SS_ERR_INVALID_ARG without touching a GPU."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    assert abs(p.gamma - 6.2831853) < 1e-6 and p.k_max == 16 and p.r_cut == 3.0
    nb = ctypes.c_size_t()
    # max_instances 0 -> invalid
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 16
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 0, ctypes.byref(nb)) == _lib.SS_ERR_INVALID_ARG
    p.max_instances = 1000
    assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 1, ctypes.byref(nb)) == 0 and nb.value > 0
    # views out of scene order, bad scene index, zero views
    d0 = _lib.ss_batch_desc(1, 0, off, cams, None)
    assert lib.ss_workspace_size(ctypes.byref(d0), ctypes.byref(p), None, 0, ctypes.byref(nb)) == _lib.SS_ERR_INVALID_ARG
    cams[0].scene = 3
    assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 0, ctypes.byref(nb)) == _lib.SS_ERR_INVALID_ARG
    cams[0].scene = 0
    p.k_max = 17
    assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 0, ctypes.byref(nb)) == _lib.SS_ERR_INVALID_ARG
    # env descriptor checks
    ed = _lib.ss_env_desc(100, 50, 6, 32, 16)
    a = ctypes.c_int64()
    assert lib.ss_env_sizes(ctypes.byref(ed), ctypes.byref(a), ctypes.byref(a), ctypes.byref(a)) == 1
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)
    b, c = ctypes.c_int64(), ctypes.c_int64()
    assert lib.ss_env_sizes(ctypes.byref(ed), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 0
    assert a.value == 32 * 16 * 3
    assert b.value == 3 * (64 * 32 + 32 * 16 + 16 * 8 + 8 * 4 * 3)
    assert lib.ss_brdf_lut(None, 128, None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_error_string(_lib.SS_ERR_CAPACITY) == b"instance capacity exceeded"
    # the launch counter is host-side: readable without a GPU, null out rejected
    n = ctypes.c_int64(-1)
    assert lib.ss_launch_count(ctypes.byref(n)) == 0 and n.value >= 0
    assert lib.ss_launch_count(None) == _lib.SS_ERR_INVALID_ARG
    # the capture query rejects a null out before any CUDA call
    assert lib.ss_stream_capture_id(None, None) == _lib.SS_ERR_INVALID_ARG


def test_launch_shape_knobs_are_validated_on_the_host():
    """Unsupported launch shapes are rejected by the host-only workspace query
    (no device pointer is involved; the render calls share the same check)."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    assert (p.fwd_warps, p.bwd_warps, p.pbwd_block) == (0, 0, 0)
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 16
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)
    nb = ctypes.c_size_t()
    assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), ctypes.byref(ed), 1, ctypes.byref(nb)) == 0
    for knob, bad, good in (("fwd_warps", 3, 4), ("bwd_warps", 1, 8), ("pbwd_block", 16, 32),
                            ("pbwd_block", 4096, 1024), ("tile_w", 12, 8), ("tile_h", 2, 4),
                            ("stage_depth", 4, 3), ("mip_mode", 3, 2), ("screen_grad", 2, 1),
                            ("deterministic", 2, 1), ("det_rows", -1, 1 << 20), ("dense_layers", 17, 2),
                            ("layer_pool", -1, 1000), ("max_candidates", -1, 1000),
                            ("zero_grad_in_forward", 2, 1)):
        q = _lib.ss_render_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        setattr(q, knob, bad)
        st = lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(q), ctypes.byref(ed), 1, ctypes.byref(nb))
        assert st == _lib.SS_ERR_INVALID_ARG, knob
        setattr(q, knob, good)
        st = lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(q), ctypes.byref(ed), 1, ctypes.byref(nb))
        assert st == 0, knob


def test_render_calls_reject_null_device_pointers():
    """The render entry points reject NULL device pointers on the host before
    anything is enqueued (no device address is ever made up here)."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 16
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    s = _lib.ss_surfels(None, None, None, None, None, None)
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)
    em = _lib.ss_env_maps(None, None, None)
    st = lib.ss_render_forward(ctypes.byref(d), ctypes.byref(s), ctypes.byref(p), ctypes.byref(ed), ctypes.byref(em),
                               None, None, None, 0, None)
    assert st == _lib.SS_ERR_INVALID_ARG
    g = _lib.ss_surfel_grads(None, None, None, None, None, None)
    st = lib.ss_render_backward(ctypes.byref(d), ctypes.byref(s), ctypes.byref(p), ctypes.byref(ed),
                                ctypes.byref(em), None, None, None, None, ctypes.byref(g), None, None, 0, None)
    assert st == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_env_prefilter(ctypes.byref(ed), 1, None, None, None, None, None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_env_prefilter_noalloc(ctypes.byref(ed), 1, None, None, None, None) == _lib.SS_ERR_INVALID_ARG
    for f in (lib.ss_env_prefilter_backward, lib.ss_env_prefilter_backward_ordered):
        assert f(ctypes.byref(ed), 1, None, None, None, None, None) == _lib.SS_ERR_INVALID_ARG


def test_tile_shapes_validated_on_the_host():
    """Tiles are unions of 8 x 4 blocks, at most 8 per tile: 32 x 16 (16 blocks)
    is refused, 8 x 32 and 32 x 8 (8 blocks) are accepted."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 40
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    nb = ctypes.c_size_t()
    for (w, h, ok) in ((32, 16, False), (32, 32, False), (8, 32, True), (32, 8, True), (8, 4, True), (16, 16, True)):
        p.tile_w, p.tile_h = w, h
        st = lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(p), None, 0, ctypes.byref(nb))
        assert (st == 0) == ok, (w, h)


def test_density_calls_validate_on_the_host():
    """Adaptive density control: struct layout, workspace sizing and the
    host-side rejections (NULL pointers, bad parameters); empty inputs are a
    no-op that launches nothing."""
    lib = _lib.lib()
    assert ctypes.sizeof(_lib.ss_density_params) == 32
    assert ctypes.sizeof(_lib.ss_stage_times) == 8 * _lib.SS_N_STAGES == 72
    p = _lib.ss_density_params()
    lib.ss_default_density(ctypes.byref(p))
    assert (p.k, p.max_rings, p.ops) == (8, 4, 7) and abs(p.split_scale - 0.7) < 1e-7 and p.cell == 0.0
    nb = ctypes.c_size_t()
    assert lib.ss_density_workspace_size(-1, ctypes.byref(nb)) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_workspace_size(10, None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_workspace_size(0, ctypes.byref(nb)) == 0 and nb.value > 0
    small = nb.value
    assert lib.ss_density_workspace_size(1_000_000, ctypes.byref(nb)) == 0 and nb.value > 40 * 1_000_000 > small
    s = _lib.ss_surfels(None, None, None, None, None, None)
    off = (ctypes.c_int64 * 2)(0, 10)
    p.cell = 0.1
    # NULL pointers with surfels to process
    assert lib.ss_density_neighbours(ctypes.byref(s), off, 1, ctypes.byref(p), None, None, None, None, 0,
                                     None) == _lib.SS_ERR_INVALID_ARG
    # bad parameters, bad offsets
    for field, bad in (("cell", 0.0), ("k", 17), ("max_rings", 0), ("ops", 9)):
        q = _lib.ss_density_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        setattr(q, field, bad)
        assert lib.ss_density_plan(None, None, None, None, None, None, 0, ctypes.byref(q), None, None, None, 0,
                                   None) == _lib.SS_ERR_INVALID_ARG, field
    bad_off = (ctypes.c_int64 * 3)(0, 10, 5)
    assert lib.ss_density_neighbours(ctypes.byref(s), bad_off, 2, ctypes.byref(p), None, None, None, None, 0,
                                     None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_plan(None, None, None, None, None, None, 5, ctypes.byref(p), None, None, None, 0,
                               None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_apply(ctypes.byref(s), 5, None, None, ctypes.c_float(0.7), ctypes.byref(s),
                                None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_apply(ctypes.byref(s), 0, None, None, ctypes.c_float(1.5), ctypes.byref(s),
                                None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_compact(None, 0, 5, None, None, 0, None, None) == _lib.SS_ERR_INVALID_ARG
    assert lib.ss_density_compact(None, 3, 5, None, None, 0, None, None) == _lib.SS_ERR_INVALID_ARG
    # nothing to do: no launch
    before = ctypes.c_int64()
    lib.ss_launch_count(ctypes.byref(before))
    zero = (ctypes.c_int64 * 2)(0, 0)
    assert lib.ss_density_neighbours(ctypes.byref(s), zero, 1, ctypes.byref(p), None, None, None, None, 0,
                                     None) == 0
    assert lib.ss_density_apply(ctypes.byref(s), 0, None, None, ctypes.c_float(0.7), ctypes.byref(s), None) == 0
    assert lib.ss_density_compact(None, 3, 0, None, None, 1, None, None) == 0
    after = ctypes.c_int64()
    lib.ss_launch_count(ctypes.byref(after))
    assert after.value == before.value


def test_deterministic_mode_sizes_its_rows_on_the_host():
    """The deterministic backward's rows (one per covering (block, surfel)
    pair: 96 bytes of sums, a record index and a list slot) are sized by
    det_rows, or by (blocks per tile) x max_instances when det_rows is 0;
    the forward-only workspace is unchanged."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 16
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)

    def size(with_bwd, **kw):
        q = _lib.ss_render_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        for k, v in kw.items():
            setattr(q, k, v)
        nb = ctypes.c_size_t()
        assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(q), ctypes.byref(ed), with_bwd,
                                     ctypes.byref(nb)) == 0
        return nb.value

    base = size(1)
    assert size(0, deterministic=1) == size(0)
    r1, r2 = size(1, deterministic=1, det_rows=10000), size(1, deterministic=1, det_rows=20000)
    assert r2 - r1 >= 10000 * 104 - 1024 and r2 - r1 <= 10000 * 104 + 1024
    # det_rows 0: (16 / 8) x (16 / 4) = 8 blocks per tile times max_instances
    assert size(1, deterministic=1) == size(1, deterministic=1, det_rows=8 * 1000) > base


def test_layer_pool_sizes_the_layer_state_on_the_host():
    """dense_layers keeps that many layers per pixel in planes of every pixel
    (13 floats each) and the deeper ones in layer_pool slots of 64 bytes: the
    workspace shrinks by (k_max - dense) planes and grows by the pool."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width, cams[0].height = 64, 32
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)

    def size(**kw):
        q = _lib.ss_render_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        for k, v in kw.items():
            setattr(q, k, v)
        nb = ctypes.c_size_t()
        assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(q), ctypes.byref(ed), 1, ctypes.byref(nb)) == 0
        return nb.value

    P = 64 * 32
    full = size()
    assert size(dense_layers=16) == full
    two = size(dense_layers=2, layer_pool=0)
    assert abs((full - two) - 14 * 13 * 4 * P) <= 512
    assert abs((size(dense_layers=2, layer_pool=5000) - two) - 5000 * 64) <= 512


def test_candidate_lists_size_the_workspace_on_the_host():
    """The rasterisers' per-block candidate and cover lists take max_candidates
    entries (4 + 8 + 4 bytes with the backward's lists), by default (blocks per
    tile) x max_instances."""
    lib = _lib.lib()
    p = _lib.ss_render_params()
    lib.ss_default_params(ctypes.byref(p))
    p.max_instances = 1000
    cams = (_lib.ss_camera * 1)()
    cams[0].width = cams[0].height = 16
    cams[0].fx = cams[0].fy = 10.0
    off = (ctypes.c_int64 * 2)(0, 10)
    d = _lib.ss_batch_desc(1, 1, off, cams, None)
    ed = _lib.ss_env_desc(64, 32, 6, 32, 16)

    def size(with_bwd, **kw):
        q = _lib.ss_render_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        for k, v in kw.items():
            setattr(q, k, v)
        nb = ctypes.c_size_t()
        assert lib.ss_workspace_size(ctypes.byref(d), ctypes.byref(q), ctypes.byref(ed), with_bwd,
                                     ctypes.byref(nb)) == 0
        return nb.value

    assert size(1) == size(1, max_candidates=8 * 1000)
    assert abs((size(1, max_candidates=20000) - size(1, max_candidates=10000)) - 10000 * 16) <= 1024
    assert abs((size(0, max_candidates=20000) - size(0, max_candidates=10000)) - 10000 * 4) <= 512
