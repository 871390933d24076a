"""Python binding of the rasterizer: the four C-ABI calls on torch tensors,
a reusable workspace holder and the torch.autograd.Function.

PyTorch supplies device memory and the stream; every step of the path runs
in libgs.so.  Functions named after the C ABI (preprocess, bin_sort,
render_fwd, render_bwd, loss_l1) only marshal arguments.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import check, lib


# ---------------------------------------------------------------- marshalling
def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def make_camera(cam) -> _lib.Camera:
    """gs_camera from an object with R, t, fx, fy, cx, cy, width, height."""
    c = _lib.Camera()
    R = np.asarray(cam.R, np.float64).reshape(9)
    t = np.asarray(cam.t, np.float64).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_config(**kw) -> _lib.Config:
    cfg = _lib.Config()
    lib().gs_config_default(C.byref(cfg))
    for k, v in kw.items():
        if k == "bg":
            for j in range(3):
                cfg.bg[j] = float(v[j])
        else:
            setattr(cfg, k, v)
    return cfg


@dataclass
class GaussianTensors:
    """Device FP32 Gaussian attributes (activated values), gs_scene layout."""
    means: torch.Tensor        # [N, 3]
    scales: torch.Tensor       # [N, 3]
    rotations: torch.Tensor    # [N, 4] (w, x, y, z)
    opacities: torch.Tensor    # [N]
    sh: torch.Tensor           # [N, K, 3]
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianTensors":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        return GaussianTensors(f(scene.means), f(scene.scales), f(scene.rotations),
                               f(scene.opacities), f(scene.sh), int(scene.sh_degree))

    def struct(self) -> _lib.Scene:
        for name in ("means", "scales", "rotations", "opacities", "sh"):
            t = getattr(self, name)
            if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        s = _lib.Scene()
        s.means, s.scales, s.rotations = self.means.data_ptr(), self.scales.data_ptr(), self.rotations.data_ptr()
        s.opacities, s.sh = self.opacities.data_ptr(), self.sh.data_ptr()
        s.n = self.n
        s.sh_degree = int(self.sh_degree)
        s.sh_coeffs = int(self.sh.shape[1])
        return s


def make_plan(n: int, cams) -> _lib.Plan:
    cam_arr = (_lib.Camera * len(cams))(*[make_camera(c) for c in cams])
    plan = _lib.Plan()
    check("gs_plan_init", lib().gs_plan_init(C.byref(plan), int(n), cam_arr, len(cams)))
    return plan


def preprocess_workspace_size(plan) -> int:
    return int(lib().gs_preprocess_workspace_size(C.byref(plan)))


def bin_sort_workspace_size(plan) -> int:
    return int(lib().gs_bin_sort_workspace_size(C.byref(plan)))


# ---------------------------------------------------------------- the C-ABI calls
def preprocess(plan, scene: _lib.Scene, cfg: _lib.Config, pre_ws: torch.Tensor,
               mask: torch.Tensor | None = None, stream=None) -> int:
    check("gs_preprocess", lib().gs_preprocess(C.byref(plan), C.byref(scene), C.byref(cfg), _ptr(mask),
                                               _ptr(pre_ws), pre_ws.numel(), _stream(stream)))
    return int(plan.n_entries)


def bin_sort(plan, pre_ws: torch.Tensor, sort_ws: torch.Tensor, stream=None) -> None:
    check("gs_bin_sort", lib().gs_bin_sort(C.byref(plan), _ptr(pre_ws), _ptr(sort_ws), sort_ws.numel(),
                                           _stream(stream)))


def render_fwd(plan, cfg, pre_ws, sort_ws, outs: dict, stream=None) -> None:
    o = _lib.FwdOutputs()
    for name, _ in _lib.FwdOutputs._fields_:
        t = outs.get(name)
        setattr(o, name, None if t is None else t.data_ptr())
    check("gs_render_fwd", lib().gs_render_fwd(C.byref(plan), C.byref(cfg), _ptr(pre_ws), _ptr(sort_ws),
                                               C.byref(o), _stream(stream)))


def render_bwd(plan, scene: _lib.Scene, cfg, pre_ws, sort_ws, dL_dimage, image, n_contrib,
               grads: dict, stream=None) -> None:
    g = _lib.Grads()
    for name, _ in _lib.Grads._fields_:
        t = grads.get(name)
        setattr(g, name, None if t is None else t.data_ptr())
    check("gs_render_bwd", lib().gs_render_bwd(C.byref(plan), C.byref(scene), C.byref(cfg), _ptr(pre_ws),
                                               _ptr(sort_ws), _ptr(dL_dimage), _ptr(image),
                                               _ptr(n_contrib), C.byref(g), _stream(stream)))


def loss_l1(image, target, loss, dL_dimage, stream=None) -> None:
    check("gs_loss_l1", lib().gs_loss_l1(_ptr(image), _ptr(target), image.numel(), _ptr(loss),
                                         _ptr(dL_dimage), _stream(stream)))


def loss_l1_ssim(plan, image, target, loss, dL_dimage, lam: float = 0.2, ws=None, l1_ssim=None,
                 stream=None) -> torch.Tensor:
    """(1 - lam) L1 + lam (1 - SSIM) and its gradient (gs_loss_l1_ssim); the
    workspace is allocated if not given.  l1_ssim: optional [2] device
    tensor receiving the two means."""
    if ws is None:
        ws = torch.empty(max(int(lib().gs_loss_l1_ssim_workspace_size(C.byref(plan))), 1), dtype=torch.uint8,
                         device=image.device)
    l1p = _ptr(l1_ssim) if l1_ssim is not None else None
    ssp = l1_ssim.data_ptr() + 4 if l1_ssim is not None else None
    check("gs_loss_l1_ssim", lib().gs_loss_l1_ssim(C.byref(plan), _ptr(image), _ptr(target), C.c_float(lam),
                                                   _ptr(loss), _ptr(dL_dimage), l1p, ssp, _ptr(ws), ws.numel(),
                                                   _stream(stream)))
    return ws


def prune_select(importance: torch.Tensor, k: int, stream=None) -> torch.Tensor:
    """Indices (ascending, int32 storage of uint32) of the k largest
    importances, ties to the lower index (gs_prune_select)."""
    n = importance.numel()
    ws = torch.empty(max(int(lib().gs_prune_workspace_size(n)), 1), dtype=torch.uint8, device=importance.device)
    keep = torch.empty(max(k, 1), dtype=torch.int32, device=importance.device)
    check("gs_prune_select", lib().gs_prune_select(_ptr(importance), n, int(k), _ptr(keep), _ptr(ws),
                                                   ws.numel(), _stream(stream)))
    return keep[:k]


ID_BLUR, ID_INTERSECT, ID_VISIBLE, ID_CRITICAL = 1, 2, 4, 8


def make_identify_config(**kw) -> _lib.ConfigIdentify:
    c = _lib.ConfigIdentify()
    lib().gs_config_identify_default(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def identify(plan, weight_sum: torch.Tensor, max_area: torch.Tensor, imax: torch.Tensor, wmax: torch.Tensor,
             cfg=None, stream=None) -> dict:
    """Per-view selections of Gaussians (gs_identify): flags [n_items] uint8
    (ID_* bits), visible_mask [n_items] uint8 (a gs_preprocess mask) and
    counts [n_views, 4] (BLUR, INTERSECT, VISIBLE, CRITICAL per view)."""
    cfg = cfg or make_identify_config()
    dev = weight_sum.device
    I = int(plan.n_items)
    flags = torch.empty(((I + 3) // 4) * 4 or 4, dtype=torch.uint8, device=dev)
    vis = torch.empty(max(I, 1), dtype=torch.uint8, device=dev)
    counts = torch.empty((int(plan.n_views), 4), dtype=torch.int32, device=dev)
    ws = torch.empty(max(int(lib().gs_identify_workspace_size(C.byref(plan))), 1), dtype=torch.uint8, device=dev)
    check("gs_identify", lib().gs_identify(C.byref(plan), C.byref(cfg), _ptr(weight_sum), _ptr(max_area), _ptr(imax),
                                           _ptr(wmax), _ptr(flags), _ptr(vis), _ptr(counts), _ptr(ws), ws.numel(),
                                           _stream(stream)))
    return {"flags": flags[:I], "visible_mask": vis[:I], "counts": counts}


def pack_mask(mask: torch.Tensor, n: int, n_views: int, stream=None) -> torch.Tensor:
    """Byte mask [n_views * n] -> the bit mask GS_FLAG_MASK_BITS reads
    (gs_pack_mask): int32 [n_views, ceil(n / 32)], bit g % 32 of word g / 32
    of row v keeps Gaussian g in view v."""
    words = (int(n) + 31) // 32
    bits = torch.empty((int(n_views), max(words, 1)), dtype=torch.int32, device=mask.device)
    check("gs_pack_mask", lib().gs_pack_mask(_ptr(mask), int(n), int(n_views), _ptr(bits), _stream(stream)))
    return bits[:, :words]


def clone_gaussians(g: "GaussianTensors", idx: torch.Tensor, stream=None) -> "GaussianTensors":
    """Aggressive clone (gs_clone_gaussians): a scene of n + k rows in which
    each Gaussian idx[r] is replaced by a clone pair (rows idx[r], n + r)."""
    n, k = g.n, int(idx.numel())
    dev = g.means.device
    out = GaussianTensors(torch.empty((n + k, 3), device=dev), torch.empty((n + k, 3), device=dev),
                          torch.empty((n + k, 4), device=dev), torch.empty((n + k,), device=dev),
                          torch.empty((n + k,) + tuple(g.sh.shape[1:]), device=dev), g.sh_degree)
    d = _lib.SceneBuf(out.means.data_ptr(), out.scales.data_ptr(), out.rotations.data_ptr(),
                      out.opacities.data_ptr(), out.sh.data_ptr(), n + k, g.sh_degree, int(g.sh.shape[1]))
    check("gs_clone_gaussians", lib().gs_clone_gaussians(C.byref(g.struct()), _ptr(idx), k, C.byref(d),
                                                         _stream(stream)))
    return out


def sample_gaussians(importance: torch.Tensor, expo: torch.Tensor, k: int, stream=None) -> torch.Tensor:
    """Primitive sampling (gs_sample_gaussians): ascending indices of k
    Gaussians drawn without replacement with P_i proportional to I_i, given
    expo ~ Exp(1); fewer if fewer have I_i > 0."""
    n = importance.numel()
    dev = importance.device
    ws = torch.empty(max(int(lib().gs_sample_workspace_size(n)), 1), dtype=torch.uint8, device=dev)
    keep = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    kk = torch.zeros(1, dtype=torch.int32, device=dev)
    check("gs_sample_gaussians", lib().gs_sample_gaussians(_ptr(importance), _ptr(expo), n, int(k), _ptr(keep),
                                                           _ptr(kk), _ptr(ws), ws.numel(), _stream(stream)))
    return keep[: int(kk.item())]


def depth_points(plan, view: int, depth: torch.Tensor, imax: torch.Tensor, target: torch.Tensor, u: torch.Tensor,
                 k: int, stream=None) -> dict:
    """Depth reinitialization seeds of one view (gs_depth_points): world
    points, colours and view-local pixel indices of k pixels drawn uniformly
    (by the largest u) among those with a contributor and d^mid > 0."""
    dev = depth.device
    ws = torch.empty(max(int(lib().gs_depth_points_workspace_size(C.byref(plan))), 1), dtype=torch.uint8,
                     device=dev)
    pts = torch.empty((max(k, 1), 3), device=dev)
    col = torch.empty((max(k, 1), 3), device=dev)
    idx = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    kk = torch.zeros(1, dtype=torch.int32, device=dev)
    check("gs_depth_points", lib().gs_depth_points(C.byref(plan), int(view), _ptr(depth), _ptr(imax),
                                                   _ptr(target), _ptr(u), int(k), _ptr(pts), _ptr(col), _ptr(idx),
                                                   _ptr(kk), _ptr(ws), ws.numel(), _stream(stream)))
    K = int(kk.item())
    return {"points": pts[:K], "colours": col[:K], "pixel_idx": idx[:K]}


def gather_scene(g: "GaussianTensors", idx: torch.Tensor, stream=None) -> "GaussianTensors":
    """A compact copy of the rows idx of every attribute (gs_gather_scene)."""
    k = int(idx.numel())
    out = GaussianTensors(torch.empty((k, 3), device=g.means.device), torch.empty((k, 3), device=g.means.device),
                          torch.empty((k, 4), device=g.means.device), torch.empty((k,), device=g.means.device),
                          torch.empty((k,) + tuple(g.sh.shape[1:]), device=g.means.device), g.sh_degree)
    if k == 0:
        return out
    d = _lib.SceneBuf(out.means.data_ptr(), out.scales.data_ptr(), out.rotations.data_ptr(),
                      out.opacities.data_ptr(), out.sh.data_ptr(), k, g.sh_degree, int(g.sh.shape[1]))
    check("gs_gather_scene", lib().gs_gather_scene(C.byref(g.struct()), _ptr(idx), k, C.byref(d), _stream(stream)))
    return out


def selftest_wait_timeout(stream=None) -> int:
    """Runs the sort's look-back wait against a predecessor that never
    publishes (gs_selftest_wait_timeout); returns the gs_status, which is
    GS_ERR_TIMEOUT when the bounded wait works."""
    ws = torch.empty(_lib.GS_SELFTEST_SCRATCH_BYTES, dtype=torch.uint8, device="cuda")
    return int(lib().gs_selftest_wait_timeout(_ptr(ws), ws.numel(), _stream(stream)))


def device_status(plan, pre_ws, stream=None) -> int:
    return int(lib().gs_device_status(C.byref(plan), _ptr(pre_ws), _stream(stream)))


def inspect_preprocess(fr: "Frame") -> dict:
    """Copies of the per-item projected state and depth order (for tests)."""
    v = _lib.PreprocessView()
    check("gs_inspect_preprocess", lib().gs_inspect_preprocess(C.byref(fr.plan), _ptr(fr.pre_ws), C.byref(v)))
    base = fr.pre_ws.data_ptr()
    I = int(fr.plan.n_items)

    def sl(ptr, count, dtype):
        off = ptr - base
        esz = torch.empty(0, dtype=dtype).element_size()
        return fr.pre_ws[off: off + count * esz].view(dtype).cpu()
    return {"xy_tau_z": sl(v.xy_tau_z, 4 * I, torch.float32).view(I, 4),
            "conic_o": sl(v.conic_o, 4 * I, torch.float32).view(I, 4),
            "rgb": sl(v.rgb, 4 * I, torch.float32).view(I, 4),
            "tiles": sl(v.tiles, I, torch.int32),
            "rect": sl(v.rect, 2 * I, torch.int32).view(I, 2),
            "sorted_items": sl(v.sorted_items, I, torch.int32),
            "offsets": sl(v.offsets, I, torch.int32),
            "pair_offsets": sl(v.pair_offsets, I, torch.int32)}


LIST_ROWS_MAX, LIST_TX_MAX = 4096, 1023


def lists_path(plan) -> bool:
    """Whether gs_bin_sort builds this plan's tile lists from (item, tile row)
    pairs (all views' tile rows at most 4096, at most 1023 tiles across any
    view) rather than by sorting the entries by tile id."""
    rows = sum((int(plan.cams[v].height) + 15) // 16 for v in range(int(plan.n_views)))
    tx = max((int(plan.cams[v].width) + 15) // 16 for v in range(int(plan.n_views)))
    return rows <= LIST_ROWS_MAX and tx <= LIST_TX_MAX


def inspect_sort(fr: "Frame") -> dict:
    """Copies of the sorted tile entries and tile ranges (for tests)."""
    v = _lib.SortView()
    check("gs_inspect_sort", lib().gs_inspect_sort(C.byref(fr.plan), _ptr(fr.sort_ws), C.byref(v)))
    base = fr.sort_ws.data_ptr()
    E, K = int(fr.plan.n_entries), int(fr.plan.total_tiles)

    def sl(ptr, count):
        off = ptr - base
        return fr.sort_ws[off: off + 4 * count].view(torch.int32).cpu()
    ranges = sl(v.ranges, 2 * K).view(K, 2)
    if v.tile_ids:
        tile_ids = sl(v.tile_ids, E)
    else:
        # the tile-list builder stores no tile id per entry: entry e belongs to
        # the tile whose range holds it
        lens = (ranges[:, 1] - ranges[:, 0]).to(torch.int64)
        tile_ids = torch.repeat_interleave(torch.arange(K, dtype=torch.int32), lens)
    return {"tile_ids": tile_ids, "items": sl(v.items, E), "ranges": ranges}


# ---------------------------------------------------------------- outputs
FWD_OUTPUTS = ("image", "final_T", "n_contrib", "imax", "wmax", "depth", "depth_blend",
               "weight_sum", "max_area", "depth_center", "n_blended")


def alloc_outputs(plan, device="cuda", want=FWD_OUTPUTS) -> dict:
    P, I = int(plan.total_pixels), int(plan.n_items)
    f32, i32 = torch.float32, torch.int32
    # weight_sum_fixed (not among the defaults): I_i in units of 2^-24 as
    # integers, bit-reproducible (unsigned 64-bit in the library, int64 here)
    spec = {"image": (3 * P, f32), "final_T": (P, f32), "n_contrib": (P, i32), "imax": (P, i32),
            "wmax": (P, f32), "depth": (P, f32), "depth_blend": (P, f32),
            "weight_sum": (I, f32), "max_area": (I, i32), "weight_sum_fixed": (I, torch.int64),
            "depth_center": (P, f32), "n_blended": (P, i32)}
    out = {}
    for k in spec:
        if k in want or k in ("image", "final_T", "n_contrib"):
            n, dt = spec[k]
            out[k] = torch.empty(max(n, 1), dtype=dt, device=device)[:n]
    for k in ("weight_sum", "max_area", "weight_sum_fixed"):
        if k in out:
            out[k].zero_()
    return out


def view_slice(plan, v: int):
    """(pixel offset, H, W) of view v in the concatenated per-pixel outputs."""
    c = plan.cams[v]
    return int(plan.pixel_base[v]), int(c.height), int(c.width)


def view_image(image: torch.Tensor, plan, v: int) -> torch.Tensor:
    off, h, w = view_slice(plan, v)
    return image[3 * off: 3 * (off + h * w)].view(3, h, w)


def view_pixels(t: torch.Tensor, plan, v: int) -> torch.Tensor:
    off, h, w = view_slice(plan, v)
    return t[off: off + h * w].view(h, w)


def alloc_grads(g: GaussianTensors) -> dict:
    z = lambda t: torch.zeros_like(t)
    return {"d_means": z(g.means), "d_scales": z(g.scales), "d_rotations": z(g.rotations),
            "d_opacities": z(g.opacities), "d_sh": z(g.sh),
            "d_mean2d_abs": torch.zeros(g.n, dtype=torch.float32, device=g.means.device)}


# ---------------------------------------------------------------- one-shot passes
@dataclass
class Frame:
    """The state of one forward pass: plan, workspaces and outputs."""
    plan: _lib.Plan
    cfg: _lib.Config
    pre_ws: torch.Tensor
    sort_ws: torch.Tensor | None
    outs: dict = field(default_factory=dict)


def forward(g: GaussianTensors, cams, cfg=None, mask=None, want=FWD_OUTPUTS, stream=None) -> Frame:
    """Preprocess, bin/sort and render every camera in one batch."""
    cfg = cfg or make_config()
    dev = g.means.device
    plan = make_plan(g.n, cams)
    pre_ws = torch.empty(preprocess_workspace_size(plan), dtype=torch.uint8, device=dev)
    preprocess(plan, g.struct(), cfg, pre_ws, mask, stream)
    sort_ws = torch.empty(bin_sort_workspace_size(plan), dtype=torch.uint8, device=dev)
    bin_sort(plan, pre_ws, sort_ws, stream)
    outs = alloc_outputs(plan, dev, want)
    render_fwd(plan, cfg, pre_ws, sort_ws, outs, stream)
    return Frame(plan, cfg, pre_ws, sort_ws, outs)


def backward(g: GaussianTensors, fr: Frame, dL_dimage: torch.Tensor, stream=None) -> dict:
    """Gradients of the attributes given dL/d image of a forward Frame.  If
    the frame's sorted lists were dropped, they are rebuilt first."""
    if fr.sort_ws is None:
        fr.sort_ws = torch.empty(bin_sort_workspace_size(fr.plan), dtype=torch.uint8, device=g.means.device)
        bin_sort(fr.plan, fr.pre_ws, fr.sort_ws, stream)
    grads = alloc_grads(g)
    render_bwd(fr.plan, g.struct(), fr.cfg, fr.pre_ws, fr.sort_ws, dL_dimage.contiguous(),
               fr.outs["image"], fr.outs["n_contrib"], grads, stream)
    return grads


class RasterizeGaussians(torch.autograd.Function):
    """Differentiable rasterization of a batch of views.

    forward(means, scales, rotations, opacities, sh, settings) returns
    (image [3 * total_pixels], depth, imax, weight_sum, max_area) where only
    the image is differentiable.  settings: RasterSettings."""

    @staticmethod
    def forward(ctx, means, scales, rotations, opacities, sh, settings):
        g = GaussianTensors(means.detach().contiguous(), scales.detach().contiguous(),
                            rotations.detach().contiguous(), opacities.detach().contiguous(),
                            sh.detach().contiguous(), settings.sh_degree)
        fr = forward(g, settings.cams, settings.cfg, settings.mask,
                     want=("image", "depth", "imax", "weight_sum", "max_area"))
        if settings.recompute_sort:
            fr.sort_ws = None          # rebuilt in backward: the lists are not kept
        ctx.frame = fr
        ctx.g = g
        o = fr.outs
        ctx.mark_non_differentiable(o["depth"], o["imax"], o["weight_sum"], o["max_area"])
        settings.last_plan = fr.plan
        return o["image"], o["depth"], o["imax"], o["weight_sum"], o["max_area"]

    @staticmethod
    def backward(ctx, d_image, *unused):
        grads = backward(ctx.g, ctx.frame, d_image)
        ctx.frame = None
        return grads["d_means"], grads["d_scales"], grads["d_rotations"], grads["d_opacities"], \
            grads["d_sh"], None


@dataclass
class RasterSettings:
    cams: list
    sh_degree: int
    cfg: _lib.Config = field(default_factory=make_config)
    mask: torch.Tensor | None = None
    recompute_sort: bool = False
    last_plan: _lib.Plan | None = None


def rasterize(means, scales, rotations, opacities, sh, settings: RasterSettings):
    return RasterizeGaussians.apply(means, scales, rotations, opacities, sh, settings)


class L1Loss(torch.autograd.Function):
    """mean |image - target| as a torch.autograd.Function over gs_loss_l1,
    which computes the loss and its gradient in one kernel; the backward
    scales the stored gradient by the incoming one."""

    @staticmethod
    def forward(ctx, image, target):
        loss = torch.zeros(1, device=image.device)
        dL = torch.empty_like(image)
        loss_l1(image.detach().contiguous(), target.detach().contiguous(), loss, dL)
        ctx.save_for_backward(dL)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dL,) = ctx.saved_tensors
        return dL * g, None


def l1_loss(image, target):
    return L1Loss.apply(image, target)
