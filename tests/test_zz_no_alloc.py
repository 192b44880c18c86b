"""The allocation-free norm, tamm_norm_noalloc, called through the C ABI.

It serves callers that must not allocate device memory while they run (their
GPU memory belongs to another allocator or pool, or an allocation would stall a
latency-critical loop).  Checked against the ordinary tamm_norm entry point on
two calls in a row, since both calls share the library's fixed scratch array.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc_norm(lib, x, n, out, stream):
    st = lib.tamm_norm_noalloc(ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(stream))
    return st


def test_noalloc_norm_matches_tamm_norm_twice(gpu_lib):
    import torch

    tg = gpu_lib
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    ctx = tg.Context(0)
    _, t = gw.build(ctx, wl.small_doubles(12, 40, 3, 5), only={"V_vvvv", "T"})
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda:0")
    for k, name in enumerate(("V_vvvv", "T")):  # two calls in a row share the scratch array
        T = t[name]
        assert _noalloc_norm(tg.load(), T.data, T.n_elems, out[k:], stream) == tg.TAMM_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k, name in enumerate(("V_vvvv", "T")):
        ref = ctx.norm(t[name])
        assert ref > 0
        assert abs(got[k] - ref) <= 1e-13 * ref, (name, got[k], ref)


def test_noalloc_norm_sizes(gpu_lib):
    import torch

    tg = gpu_lib
    lib = tg.load()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
    # more than one partial block, ragged end
    x = torch.arange(1, 40001, dtype=torch.float64, device="cuda:0")
    assert _noalloc_norm(lib, x, x.numel(), out, stream) == tg.TAMM_OK
    torch.cuda.synchronize()
    n = 40000
    ref = np.sqrt(n * (n + 1) * (2 * n + 1) / 6)
    assert abs(out.item() - ref) <= 1e-14 * ref
    # empty input gives 0
    assert _noalloc_norm(lib, x, 0, out, stream) == tg.TAMM_OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # sizes past the fixed scratch are refused before any launch
    assert lib.tamm_norm_noalloc(ctypes.c_void_p(x.data_ptr()), (1 << 29) + 1, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream)) == tg.TAMM_ELIMIT
    assert lib.tamm_norm_noalloc(ctypes.c_void_p(x.data_ptr()), -1, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream)) == tg.TAMM_EINVAL
    # pointers that are not 8-byte aligned are refused before any launch
    assert lib.tamm_norm_noalloc(ctypes.c_void_p(x.data_ptr() + 4), 8, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream)) == tg.TAMM_EINVAL
    assert lib.tamm_norm_noalloc(ctypes.c_void_p(x.data_ptr()), 8, ctypes.c_void_p(out.data_ptr() + 4),
                                 ctypes.c_void_p(stream)) == tg.TAMM_EINVAL
