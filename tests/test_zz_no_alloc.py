"""gs_bin_sort_noalloc: binning and tile sort without any device allocation.

This entry point serves callers that cannot allocate GPU memory when they
render (for example a host application that owns all device memory and only
hands out fixed buffers).  They pass the output arrays; the sort's scratch
comes from a fixed device array inside the library.  Its results must equal
those of gs_bin_sort, which sorts in a caller-allocated workspace: tile ids,
items and tile ranges are integers, so the comparison is bit-exact.  Two
different scenes are binned back to back (and the first again) so that
state left in the shared scratch by one call cannot leak into the next.

This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_12788_gb300 import _lib, raster, scenes

pytestmark = pytest.mark.gpu


def _cases():
    def multiview():
        cams = []
        for (w, h), e in zip([(50, 37), (64, 64), (33, 20)], [(0, 0, 0), (0.4, -0.2, 0.3), (-0.5, 0.3, -0.2)]):
            cams.append(scenes.fov_camera(*scenes.look_at(e, (0, 0, 4.0)), w, h, 50.0))
        return scenes.box_scene(512, seed=4, sh_degree=3), cams
    return [
        (scenes.box_scene(1024, seed=0), [scenes.origin_camera()]),
        multiview(),
        (scenes.cluster_scene(60_000, 64, seed=3, sh_degree=1), [scenes.ring_camera(0.5, 640, 480)]),
        # 320 tiles: the tile-id sort is one pass of 512 digits, copied back
        # out of the alternate buffers (the other cases sort 4 or 11 bits)
        (scenes.cluster_scene(30_000, 32, seed=5, sh_degree=1), [scenes.ring_camera(0.2, 320, 256)]),
    ]


def _noalloc(fr):
    E, K = int(fr.plan.n_entries), int(fr.plan.total_tiles)
    tile_ids = torch.full((max(E, 1),), -1, dtype=torch.int32, device="cuda")
    items = torch.full((max(E, 1),), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((K, 2), -1, dtype=torch.int32, device="cuda")
    st = _lib.lib().gs_bin_sort_noalloc(C.byref(fr.plan), C.c_void_p(fr.pre_ws.data_ptr()),
                                        C.c_void_p(tile_ids.data_ptr()), C.c_void_p(items.data_ptr()),
                                        C.c_void_p(ranges.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.STATUS.get(st, st)
    torch.cuda.synchronize()
    return tile_ids[:E].cpu(), items[:E].cpu(), ranges.cpu()


def test_noalloc_matches_bin_sort_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = _cases()
    for sc, cams in cases + cases[:1]:
        g = raster.GaussianTensors.from_scene(sc)
        fr = raster.forward(g, cams)          # gs_bin_sort with a caller workspace
        assert 0 < fr.plan.n_entries <= (1 << 19)
        ref = raster.inspect_sort(fr)
        t, i, r = _noalloc(fr)
        assert torch.equal(t, ref["tile_ids"])
        assert torch.equal(i, ref["items"])
        assert torch.equal(r, ref["ranges"])
        assert raster.device_status(fr.plan, fr.pre_ws) == 0


def test_noalloc_rejects_more_entries_than_its_scratch_holds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc, cams = _cases()[0]
    fr = raster.forward(raster.GaussianTensors.from_scene(sc), cams)
    plan = _lib.Plan()
    C.memmove(C.byref(plan), C.byref(fr.plan), C.sizeof(plan))
    plan.n_entries = (1 << 19) + 1
    dummy = torch.empty(4, dtype=torch.int32, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = _lib.lib().gs_bin_sort_noalloc(C.byref(plan), C.c_void_p(fr.pre_ws.data_ptr()), p, p, p, None)
    assert st == 2          # GS_ERR_CAPACITY, before anything is launched
