"""The environment prefilter entry point for callers that cannot allocate
device memory (plugins handed only input/output buffers, code under a fixed
budget or an allocator that forbids cudaMalloc) must give the same maps as
the allocating entry point, on consecutive calls.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _maps(lib, desc, n_envs, env, noalloc):
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import _ptr, _stream
    ni, ns, na = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _lib.check(lib.ss_env_sizes(ctypes.byref(desc), ctypes.byref(ni), ctypes.byref(ns), ctypes.byref(na)))
    irr = torch.full((n_envs, ni.value), -1.0, device="cuda")
    spec = torch.full((n_envs, ns.value), -1.0, device="cuda")
    if noalloc:
        st = lib.ss_env_prefilter_noalloc(ctypes.byref(desc), n_envs, _ptr(env), _ptr(irr), _ptr(spec), _stream())
    else:
        aux = torch.zeros(n_envs, na.value, device="cuda")
        st = lib.ss_env_prefilter(ctypes.byref(desc), n_envs, _ptr(env), _ptr(irr), _ptr(spec), _ptr(aux), _stream())
    _lib.check(st, "prefilter")
    torch.cuda.synchronize()
    return irr.cpu().numpy(), spec.cpu().numpy()


def test_noalloc_prefilter_matches_allocating_entry_on_two_calls():
    import torch
    from paper_2605_05876_gb300 import _lib, build
    build()
    lib = _lib.lib()
    rng = np.random.default_rng(77)
    # two calls in a row with different maps and sizes; the shared scratch
    # keeps the first call's contents when the second one runs
    for (We, He, L, n_envs) in [(256, 128, 6, 3), (64, 32, 5, 2)]:
        env = torch.from_numpy(np.exp(rng.normal(size=(n_envs, He, We, 3))).astype(np.float32)).cuda()
        desc = _lib.ss_env_desc(We, He, L, 32, 16)
        ref_irr, ref_spec = _maps(lib, desc, n_envs, env, noalloc=False)
        got_irr, got_spec = _maps(lib, desc, n_envs, env, noalloc=True)
        # the same deterministic kernels on the same inputs: equal bit for bit
        assert np.array_equal(got_irr, ref_irr)
        assert np.array_equal(got_spec, ref_spec)


def test_noalloc_prefilter_rejects_sizes_beyond_its_scratch():
    """A map whose scratch exceeds the fixed array is refused with
    SS_ERR_INVALID_ARG; the buffers passed are real and correctly sized, so a
    regression in the size check would give a wrong status, not a fault, and
    the outputs must be left untouched."""
    import torch
    from paper_2605_05876_gb300 import _lib, build
    from paper_2605_05876_gb300.api import _ptr, _stream
    build()
    lib = _lib.lib()
    desc = _lib.ss_env_desc(2048, 1024, 6, 32, 16)   # aux of one map exceeds the fixed scratch
    ni, ns, na = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert lib.ss_env_sizes(ctypes.byref(desc), ctypes.byref(ni), ctypes.byref(ns), ctypes.byref(na)) == 0
    assert na.value > _lib.SS_NOALLOC_AUX_FLOATS
    env = torch.ones(1, 1024, 2048, 3, device="cuda")
    irr = torch.full((1, ni.value), -1.0, device="cuda")
    spec = torch.full((1, ns.value), -1.0, device="cuda")
    st = lib.ss_env_prefilter_noalloc(ctypes.byref(desc), 1, _ptr(env), _ptr(irr), _ptr(spec), _stream())
    assert st == _lib.SS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((irr == -1.0).all()) and bool((spec == -1.0).all())
