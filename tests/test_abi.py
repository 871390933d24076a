"""The C ABI without a GPU: the library loads, exports every function that
include/gs.h declares, its struct layouts match the binding, and host-side
argument validation rejects bad calls before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2411_12788_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_functions_are_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    from paper_2411_12788_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_header_constants_match_the_binding():
    """Every #define of include/gs.h that the Python binding also names has
    the same value there."""
    from paper_2411_12788_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    defs = dict(re.findall(r"#define\s+(GS_[A-Z0-9_]+)\s+\(?([0-9]+)u?\)?", src))
    shared = [k for k in defs if hasattr(_lib, k)]
    assert {"GS_FLAG_ZERO_ACCUM", "GS_FLAG_EXTENT_3SIGMA", "GS_TILE"} <= set(shared)
    for k in shared:
        assert getattr(_lib, k) == int(defs[k]), k


def test_struct_sizes(L):
    from paper_2411_12788_gb300 import _lib
    assert L.gs_sizeof_plan() == C.sizeof(_lib.Plan)
    assert L.gs_sizeof_camera() == C.sizeof(_lib.Camera) == 72
    assert L.gs_sizeof_config() == C.sizeof(_lib.Config)
    assert L.gs_sizeof_scene() == C.sizeof(_lib.Scene)


def _cam(w=64, h=48, f=50.0):
    from paper_2411_12788_gb300 import _lib
    c = _lib.Camera()
    for k in range(9):
        c.R[k] = 1.0 if k in (0, 4, 8) else 0.0
    c.fx = c.fy = f
    c.cx, c.cy = w / 2, h / 2
    c.width, c.height = w, h
    return c


def test_plan_init_and_validation(L):
    from paper_2411_12788_gb300 import _lib
    plan = _lib.Plan()
    cams = (_lib.Camera * 3)(_cam(50, 37), _cam(64, 64), _cam(33, 20))
    assert L.gs_plan_init(C.byref(plan), 1000, cams, 3) == 0
    assert plan.n_items == 3000
    assert plan.total_tiles == 4 * 3 + 4 * 4 + 3 * 2
    assert list(plan.tile_base)[:4] == [0, 12, 28, 34]
    assert list(plan.pixel_base)[:4] == [0, 1850, 1850 + 4096, 1850 + 4096 + 660]
    assert plan.total_pixels == 1850 + 4096 + 660
    assert plan.sort_bits == 6                     # 34 tiles -> 6 bits
    assert plan.n_entries == -1
    assert L.gs_preprocess_workspace_size(C.byref(plan)) > 3000 * 150
    assert L.gs_bin_sort_workspace_size(C.byref(plan)) == 0      # before preprocess
    assert L.gs_plan_init(C.byref(plan), 10, cams, 0) == 1
    assert L.gs_plan_init(C.byref(plan), 10, cams, 65) == 1
    assert L.gs_plan_init(C.byref(plan), -1, cams, 1) == 1
    bad = (_lib.Camera * 1)(_cam(0, 10))
    assert L.gs_plan_init(C.byref(plan), 10, bad, 1) == 1
    bad = (_lib.Camera * 1)(_cam(10, 10, f=0.0))
    assert L.gs_plan_init(C.byref(plan), 10, bad, 1) == 1
    assert L.gs_plan_init(C.byref(plan), 1 << 29, (_lib.Camera * 2)(_cam(), _cam()), 2) == 1


def test_host_side_argument_checks(L):
    """Calls that must fail before touching the device (no GPU needed)."""
    from paper_2411_12788_gb300 import _lib
    plan = _lib.Plan()
    cams = (_lib.Camera * 1)(_cam())
    assert L.gs_plan_init(C.byref(plan), 100, cams, 1) == 0
    cfg = _lib.Config()
    L.gs_config_default(C.byref(cfg))
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and cfg.alpha_max == pytest.approx(0.99)
    fake = 1 << 20                                  # aligned non-null stand-in, never dereferenced
    sc = _lib.Scene(fake, fake, fake, fake, fake, 100, 3, 16)
    ws_need = L.gs_preprocess_workspace_size(C.byref(plan))
    # null scene, degree out of range, wrong n, too few SH columns, misaligned rotations
    assert L.gs_preprocess(C.byref(plan), None, C.byref(cfg), None, fake, ws_need, None) == 1
    for kw in (dict(sh_degree=4), dict(n=99), dict(sh_coeffs=15), dict(rotations=fake + 4)):
        s2 = _lib.Scene(fake, fake, fake, fake, fake, 100, 3, 16)
        for k, v in kw.items():
            setattr(s2, k, v)
        assert L.gs_preprocess(C.byref(plan), C.byref(s2), C.byref(cfg), None, fake, ws_need, None) == 1, kw
    bad = _lib.Config()
    L.gs_config_default(C.byref(bad))
    bad.alpha_max = 1.5
    assert L.gs_preprocess(C.byref(plan), C.byref(sc), C.byref(bad), None, fake, ws_need, None) == 1
    # misaligned and too-small workspaces
    assert L.gs_preprocess(C.byref(plan), C.byref(sc), C.byref(cfg), None, fake + 16, ws_need, None) == 1
    assert L.gs_preprocess(C.byref(plan), C.byref(sc), C.byref(cfg), None, fake, ws_need - 1, None) == 2
    # calls that need a completed preprocess
    out = _lib.FwdOutputs()
    assert L.gs_render_fwd(C.byref(plan), C.byref(cfg), fake, fake, C.byref(out), None) == 1
    assert L.gs_bin_sort(C.byref(plan), fake, fake, 1 << 30, None) == 1
    assert L.gs_loss_l1(None, fake, 10, fake, fake, None) == 1
    assert L.gs_status_string(2) == b"workspace too small"


def _paper_constants():
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_identify_defaults_are_the_papers_constants(L):
    """The identification defaults of the library and of the oracle are the
    values the paper prints (Sec. 4.1 theta_blur, Sec. 5.1 and 5.2 keep
    quantiles; tests/golden/paper_constants.txt)."""
    import inspect

    import numpy as np

    from oracle import identify as OI
    from paper_2411_12788_gb300 import _lib
    paper = _paper_constants()
    assert set(paper) == {"theta_blur", "keep_critical", "keep_visible"}
    cfg = _lib.ConfigIdentify()
    L.gs_config_identify_default(C.byref(cfg))
    for name in paper:
        assert getattr(cfg, name) == np.float32(paper[name]), name
    assert inspect.signature(OI.blur_split).parameters["theta"].default == paper["theta_blur"]
    assert inspect.signature(OI.visible).parameters["q"].default == paper["keep_visible"]
