"""The checked build (GS_CHECKED, libgs_checked.so): every computed index into
an entry, item or output array is checked before the access, and an
out-of-range one is recorded in the device status word (gs_device_status then
returns GS_ERR_DEVICE_CHECK) and skipped instead of faulting.  On the parity
scenes and a training-scale scene the checked build records nothing and
computes what the normal build computes: the same images, contribution counts
and i_max, and the same gradients up to the order of the float atomics.

The checked library runs in a child process (the binding picks the library
when it is imported, from GS_CHECKED)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2411_12788_gb300 import build, raster, scenes

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2411_12788_gb300 import _lib, raster, scenes
assert _lib.LIB_PATH.endswith("libgs_checked.so")
out = sys.argv[2]
import importlib.util
spec = importlib.util.spec_from_file_location("cases", sys.argv[3])
cases = importlib.util.module_from_spec(spec); spec.loader.exec_module(cases)
for name, res in cases.run_all():
    np.savez(f"{out}/{name}.npz", **res)
"""


def run_all():
    """(name, arrays) for every case: forward outputs, the device status after
    forward and backward, and the attribute gradients of an L1 loss."""
    cams_mv = []
    for (w, h), e in zip([(50, 37), (64, 64), (33, 20)], [(0, 0, 0), (0.4, -0.2, 0.3), (-0.5, 0.3, -0.2)]):
        cams_mv.append(scenes.fov_camera(*scenes.look_at(e, (0, 0, 4.0)), w, h, 50.0))
    cases = [("box1024", scenes.box_scene(1024, seed=0), [scenes.origin_camera()]),
             ("multiview", scenes.box_scene(512, seed=4, sh_degree=3), cams_mv),
             ("cluster200k", scenes.cluster_scene(200_000, 64, seed=0, sh_degree=3),
              [scenes.ring_camera(0.3, 1600, 1063), scenes.ring_camera(2.0, 800, 800)])]
    for name, sc, cams in cases:
        g = raster.GaussianTensors.from_scene(sc)
        fr = raster.forward(g, cams)
        dL = torch.sign(fr.outs["image"] - 0.5) / fr.outs["image"].numel()
        grads = raster.backward(g, fr, dL)
        torch.cuda.synchronize()
        res = {k: fr.outs[k].cpu().numpy() for k in ("image", "n_contrib", "imax", "final_T")}
        res.update({k: v.cpu().numpy() for k, v in grads.items()})
        res["status"] = np.array([raster.device_status(fr.plan, fr.pre_ws)])
        res["n_entries"] = np.array([int(fr.plan.n_entries)])
        yield name, res


def test_checked_build_records_nothing_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build(checked=True)
    env = dict(os.environ, GS_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path), os.path.abspath(__file__)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    for name, ref in run_all():
        got = np.load(tmp_path / f"{name}.npz")
        assert int(got["status"][0]) == 0 and int(ref["status"][0]) == 0, name
        assert int(got["n_entries"][0]) == int(ref["n_entries"][0]) > 0, name
        for k in ("image", "n_contrib", "imax", "final_T"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{name} {k}")
        # gradients: equal up to the order of the float atomics, which moves
        # sums with cancellation by a few 1e-5 of the tensor's largest entry
        for k in ("d_means", "d_scales", "d_rotations", "d_opacities", "d_sh"):
            a, b = got[k].astype(np.float64), ref[k].astype(np.float64)
            tol = 2e-4 * np.abs(b).max() + 1e-12
            assert np.abs(a - b).max() <= tol, (name, k, np.abs(a - b).max(), tol)
