"""Thin ctypes binding of libgs3dtr.so (C ABI declared in include/gs3dtr.h).

Only argument marshalling lives here: every step of the iteration runs in the
CUDA library.  Functions keep the C names; tensors are torch CUDA tensors whose
device pointers are passed through, and the stream is torch's current stream
unless one is given.  If the library has not been built, loading fails loudly:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs3dtr.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_UNSUPPORTED = 0, 1, 2, 3
GS_FLAG_CAPACITY, GS_FLAG_NONFINITE, GS_FLAG_TIMEOUT = 1, 2, 4
GS_LOSS_L1, GS_LOSS_L2, GS_LOSS_COTANGENT, GS_LOSS_WEIGHTED = 0, 1, 2, 3

EXPORTED = ("gs_last_error", "gs_version", "gs_project", "gs_bin_sort_workspace_size", "gs_bin_sort",
            "gs_bin_sort_noalloc",
            "gs_raster_fwd", "gs_raster_bwd_workspace_size", "gs_raster_bwd", "gs_hvp_diag", "gs_tr_update",
            "gs_tr_update_dev", "gs_step_advance", "gs_adam_tr_update", "gs_dssim_workspace_size",
            "gs_dssim_cotangents", "gs_wait_check", "gs_project_batch", "gs_raster_bwd_batch", "gs_tr_update_batch")


class gs_params(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_pad", C.c_int32), ("sh_degree", C.c_int32), ("reserved", C.c_int32),
                ("data", C.c_void_p)]


class gs_camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("near_plane", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("reserved", C.c_int32)]


class gs_frame(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("footprint_bins", C.c_int32), ("batch", C.c_int32)]


class gs_probe(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("t", C.c_int64), ("nu", C.c_int32), ("reserved", C.c_int32),
                ("t_device", C.c_void_p)]


class gs_eps_schedule(C.Structure):
    _fields_ = [("eps0", C.c_double), ("eps1", C.c_double), ("total", C.c_int64)]


class gs_adam_config(C.Structure):
    _fields_ = [("beta1", C.c_float), ("beta2", C.c_float), ("eps_adam", C.c_float), ("lr", C.c_float * 6)]


def adam_struct(beta1=0.9, beta2=0.999, eps_adam=1e-15, lr=(1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4)):
    """Adam hyper-parameters; learning rates of the row groups mean, log-scale,
    quaternion, opacity logit, SH DC, other SH."""
    return gs_adam_config(beta1, beta2, eps_adam, (C.c_float * 6)(*lr))


class gs_projected(C.Structure):
    _fields_ = [("rec", C.c_void_p), ("tangent", C.c_void_p)]


class gs_sorted(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("vals", C.c_void_p), ("ranges", C.c_void_p), ("n_pairs", C.c_void_p),
                ("capacity", C.c_uint64), ("order", C.c_void_p), ("masks", C.c_void_p)]


class gs_loss(C.Structure):
    _fields_ = [("kind", C.c_int32), ("gn_floor", C.c_float)]


class gs_tr_config(C.Structure):
    _fields_ = [("theta1", C.c_float), ("theta2", C.c_float), ("d_floor", C.c_float), ("color_floor", C.c_float),
                ("l", C.c_int32), ("mean_exact", C.c_int32)]


GS_BATCH_MAX = 16


class gs_batch_item(C.Structure):
    _fields_ = [("x", gs_params), ("grad", gs_params), ("hz", gs_params), ("g_ema", gs_params), ("d_ema", gs_params),
                ("cam", C.c_void_p), ("t", C.c_int64), ("eps", C.c_float), ("hvp", C.c_int32)]


assert C.sizeof(gs_camera) == 96 and C.sizeof(gs_params) == 24 and C.sizeof(gs_sorted) == 56
assert C.sizeof(gs_batch_item) == 144


class GSError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None


def load():
    """Load libgs3dtr.so; raises if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise GSError(f"{LIB_PATH} is missing: build it with paper_2602_00395_gb300.build.build() "
                          "(the CUDA library is the only implementation)")
        L = C.CDLL(LIB_PATH)
        P, st = C.c_void_p, C.c_int32
        i32p = C.POINTER(C.c_int32)
        L.gs_last_error.restype = C.c_char_p
        L.gs_version.restype = C.c_int32
        L.gs_project.restype = st
        L.gs_project.argtypes = [C.POINTER(gs_params), P, gs_frame, C.POINTER(gs_probe), C.POINTER(gs_projected),
                                 P, P]
        L.gs_bin_sort_workspace_size.restype = C.c_size_t
        L.gs_bin_sort_workspace_size.argtypes = [C.c_int32, gs_frame, C.c_uint64]
        L.gs_bin_sort.restype = st
        L.gs_bin_sort.argtypes = [C.POINTER(gs_projected), C.c_int32, gs_frame, P, C.c_size_t,
                                  C.POINTER(gs_sorted), P, P]
        L.gs_bin_sort_noalloc.restype = st
        L.gs_bin_sort_noalloc.argtypes = [C.POINTER(gs_projected), C.c_int32, gs_frame, C.POINTER(gs_sorted), P, P]
        L.gs_raster_fwd.restype = st
        L.gs_raster_fwd.argtypes = [C.POINTER(gs_projected), C.POINTER(gs_sorted), C.c_int32, gs_frame,
                                    C.POINTER(gs_probe), P, P, P, P, P, P]
        L.gs_raster_bwd_workspace_size.restype = C.c_size_t
        L.gs_raster_bwd_workspace_size.argtypes = [C.c_int32, gs_frame, C.c_int32]
        L.gs_raster_bwd.restype = st
        L.gs_raster_bwd.argtypes = [C.POINTER(gs_params), P, gs_frame, C.POINTER(gs_projected),
                                    C.POINTER(gs_sorted), P, P, P, P, P, C.POINTER(gs_probe), gs_loss,
                                    C.POINTER(gs_params), C.POINTER(gs_params), P, P, C.c_size_t, P, P]
        L.gs_hvp_diag.restype = st
        L.gs_hvp_diag.argtypes = [C.POINTER(gs_params), P, gs_frame, C.POINTER(gs_projected), C.POINTER(gs_sorted),
                                  P, P, P, P, P, C.POINTER(gs_probe), gs_loss, C.POINTER(gs_params), P, C.c_size_t,
                                  P, P]
        L.gs_tr_update.restype = st
        L.gs_tr_update.argtypes = [C.POINTER(gs_params), C.POINTER(gs_params), C.POINTER(gs_params),
                                   C.POINTER(gs_params), C.POINTER(gs_params), C.POINTER(gs_tr_config), C.c_int64,
                                   C.c_float, C.POINTER(gs_params), P, P]
        L.gs_tr_update_dev.restype = st
        L.gs_tr_update_dev.argtypes = [C.POINTER(gs_params), C.POINTER(gs_params), C.POINTER(gs_params),
                                       C.POINTER(gs_params), C.POINTER(gs_params), C.POINTER(gs_tr_config), P,
                                       C.POINTER(gs_eps_schedule), C.POINTER(gs_params), P, P]
        L.gs_step_advance.restype = st
        L.gs_step_advance.argtypes = [P, P]
        L.gs_wait_check.restype = st
        L.gs_wait_check.argtypes = [C.c_uint32, P, P]
        L.gs_dssim_workspace_size.restype = C.c_size_t
        L.gs_dssim_workspace_size.argtypes = [gs_frame, C.c_int32]
        L.gs_dssim_cotangents.restype = st
        L.gs_dssim_cotangents.argtypes = [gs_frame, P, P, P, C.c_int32, C.c_float, C.c_float, C.c_int32, P, P, P,
                                          C.c_size_t, P, P]
        BI = C.POINTER(gs_batch_item)
        L.gs_project_batch.restype = st
        L.gs_project_batch.argtypes = [BI, C.c_int32, C.c_int32, gs_frame, C.POINTER(gs_probe),
                                       C.POINTER(gs_projected), P, P]
        L.gs_raster_bwd_batch.restype = st
        L.gs_raster_bwd_batch.argtypes = [BI, C.c_int32, C.c_int32, gs_frame, C.POINTER(gs_projected),
                                          C.POINTER(gs_sorted), P, P, P, P, P, C.POINTER(gs_probe), gs_loss, P, P,
                                          C.c_size_t, P, P]
        L.gs_tr_update_batch.restype = st
        L.gs_tr_update_batch.argtypes = [BI, C.c_int32, C.POINTER(gs_tr_config), P, P]
        L.gs_adam_tr_update.restype = st
        L.gs_adam_tr_update.argtypes = [C.POINTER(gs_params), C.POINTER(gs_params), C.POINTER(gs_params),
                                        C.POINTER(gs_params), C.POINTER(gs_tr_config), C.POINTER(gs_adam_config),
                                        C.c_int64, C.c_float, C.POINTER(gs_params), P, P]
        _lib = L
        return L


def check(code: int, what: str = "") -> None:
    if code != GS_OK:
        msg = load().gs_last_error().decode(errors="replace")
        raise GSError(f"{what or 'gs call'} failed with status {code}: {msg}")


# ------------------------------------------------------------ marshalling
def ptr(t) -> int | None:
    """Device pointer of a tensor (None passes NULL)."""
    return None if t is None else t.data_ptr()


def stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def params_struct(data, n: int, sh_degree: int) -> gs_params:
    """gs_params over a float32 CUDA tensor of shape [rows, n_pad]."""
    assert data.dtype.is_floating_point and data.dim() == 2 and data.is_contiguous()
    return gs_params(n, data.shape[1], sh_degree, 0, data.data_ptr())


def camera_bytes(cams) -> np.ndarray:
    """Pack cameras (objects with viewmat, fx, fy, cx, cy, near, width, height) as gs_camera structs."""
    arr = (gs_camera * len(cams))()
    for k, c in enumerate(cams):
        vm = np.asarray(c.viewmat, np.float64).reshape(16)
        arr[k].viewmat[:] = [float(v) for v in vm]
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = c.fx, c.fy, c.cx, c.cy
        arr[k].near_plane = c.near
        arr[k].width, arr[k].height = c.width, c.height
    return np.frombuffer(bytes(arr), np.uint8).copy()


def frame_struct(n_views: int, width: int, height: int, tile_w: int = 16, tile_h: int = 16,
                 footprint_bins: bool = True, batch: int = 0) -> gs_frame:
    return gs_frame(n_views, width, height, tile_w, tile_h, int(footprint_bins), int(batch))


def probe_struct(seed: int, t: int, nu: int, t_device=None) -> gs_probe:
    """Probe descriptor; t_device (a device int64 tensor) makes the kernels read
    the step index from device memory (for calls captured in a CUDA graph)."""
    return gs_probe(seed, t, nu, 0, ptr(t_device) if t_device is not None else None)


# ------------------------------------------------------------ the six calls
def gs_project(x: gs_params, cams_dev, frame: gs_frame, probe: gs_probe | None, out: gs_projected,
               status=None, stream=None) -> None:
    L = load()
    check(L.gs_project(C.byref(x), ptr(cams_dev), frame, C.byref(probe) if probe else None, C.byref(out),
                       ptr(status), stream_handle(stream)), "gs_project")


def gs_bin_sort_workspace_size(n_pad: int, frame: gs_frame, capacity: int) -> int:
    return int(load().gs_bin_sort_workspace_size(n_pad, frame, capacity))


def gs_bin_sort(proj: gs_projected, n_pad: int, frame: gs_frame, workspace, out: gs_sorted, status=None,
                stream=None) -> None:
    L = load()
    check(L.gs_bin_sort(C.byref(proj), n_pad, frame, ptr(workspace), workspace.numel() * workspace.element_size(),
                        C.byref(out), ptr(status), stream_handle(stream)), "gs_bin_sort")


def gs_bin_sort_noalloc(proj: gs_projected, n_pad: int, frame: gs_frame, out: gs_sorted, status=None,
                        stream=None) -> None:
    """gs_bin_sort without a caller workspace (the library's fixed 32 MiB scratch)."""
    L = load()
    check(L.gs_bin_sort_noalloc(C.byref(proj), n_pad, frame, C.byref(out), ptr(status), stream_handle(stream)),
          "gs_bin_sort_noalloc")


def gs_raster_fwd(proj: gs_projected, sorted_: gs_sorted, n_pad: int, frame: gs_frame, probe: gs_probe | None,
                  image, final_T, n_contrib, image_tangent=None, status=None, stream=None) -> None:
    L = load()
    check(L.gs_raster_fwd(C.byref(proj), C.byref(sorted_), n_pad, frame, C.byref(probe) if probe else None,
                          ptr(image), ptr(final_T), ptr(n_contrib), ptr(image_tangent), ptr(status),
                          stream_handle(stream)), "gs_raster_fwd")


def gs_raster_bwd_workspace_size(n_pad: int, frame: gs_frame, nu: int) -> int:
    return int(load().gs_raster_bwd_workspace_size(n_pad, frame, nu))


def gs_raster_bwd(x: gs_params, cams_dev, frame: gs_frame, proj: gs_projected, sorted_: gs_sorted, image, target,
                  final_T, n_contrib, image_tangent, probe: gs_probe | None, loss: gs_loss, grad: gs_params,
                  hz: gs_params | None, loss_out, workspace, status=None, stream=None) -> None:
    L = load()
    check(L.gs_raster_bwd(C.byref(x), ptr(cams_dev), frame, C.byref(proj), C.byref(sorted_), ptr(image), ptr(target),
                          ptr(final_T), ptr(n_contrib), ptr(image_tangent), C.byref(probe) if probe else None, loss,
                          C.byref(grad), C.byref(hz) if hz else None, ptr(loss_out), ptr(workspace),
                          workspace.numel() * workspace.element_size(), ptr(status), stream_handle(stream)),
          "gs_raster_bwd")


def gs_hvp_diag(x: gs_params, cams_dev, frame: gs_frame, proj: gs_projected, sorted_: gs_sorted, image, target,
                final_T, n_contrib, image_tangent, probe: gs_probe, loss: gs_loss, hz: gs_params, workspace,
                status=None, stream=None) -> None:
    L = load()
    check(L.gs_hvp_diag(C.byref(x), ptr(cams_dev), frame, C.byref(proj), C.byref(sorted_), ptr(image), ptr(target),
                        ptr(final_T), ptr(n_contrib), ptr(image_tangent), C.byref(probe), loss, C.byref(hz),
                        ptr(workspace), workspace.numel() * workspace.element_size(), ptr(status),
                        stream_handle(stream)), "gs_hvp_diag")


def gs_tr_update(x: gs_params, g_ema: gs_params, d_ema: gs_params, grad: gs_params, hz: gs_params | None,
                 cfg: gs_tr_config, t: int, eps: float, eta_out: gs_params | None = None, status=None,
                 stream=None) -> None:
    L = load()
    check(L.gs_tr_update(C.byref(x), C.byref(g_ema), C.byref(d_ema), C.byref(grad), C.byref(hz) if hz else None,
                         C.byref(cfg), t, eps, C.byref(eta_out) if eta_out else None, ptr(status),
                         stream_handle(stream)), "gs_tr_update")


def gs_tr_update_dev(x: gs_params, g_ema: gs_params, d_ema: gs_params, grad: gs_params, hz: gs_params | None,
                     cfg: gs_tr_config, t_device, schedule: gs_eps_schedule, eta_out: gs_params | None = None,
                     status=None, stream=None) -> None:
    L = load()
    check(L.gs_tr_update_dev(C.byref(x), C.byref(g_ema), C.byref(d_ema), C.byref(grad),
                             C.byref(hz) if hz else None, C.byref(cfg), ptr(t_device), C.byref(schedule),
                             C.byref(eta_out) if eta_out else None, ptr(status), stream_handle(stream)),
          "gs_tr_update_dev")


def gs_step_advance(t_device, stream=None) -> None:
    L = load()
    check(L.gs_step_advance(ptr(t_device), stream_handle(stream)), "gs_step_advance")


def gs_wait_check(limit: int, status, stream=None) -> None:
    L = load()
    check(L.gs_wait_check(limit, ptr(status), stream_handle(stream)), "gs_wait_check")


def gs_adam_tr_update(x: gs_params, m: gs_params, v: gs_params, grad: gs_params, cfg: gs_tr_config,
                      adam: gs_adam_config, t: int, eps: float, eta_out: gs_params | None = None, status=None,
                      stream=None) -> None:
    L = load()
    check(L.gs_adam_tr_update(C.byref(x), C.byref(m), C.byref(v), C.byref(grad), C.byref(cfg), C.byref(adam), t,
                              eps, C.byref(eta_out) if eta_out else None, ptr(status), stream_handle(stream)),
          "gs_adam_tr_update")


def gs_dssim_workspace_size(frame: gs_frame, nu: int) -> int:
    return int(load().gs_dssim_workspace_size(frame, nu))


def gs_dssim_cotangents(frame: gs_frame, image, target, image_tangent, nu: int, lam: float, gn_floor: float,
                        want_grad: bool, cot, loss_out, workspace, status=None, stream=None) -> None:
    L = load()
    check(L.gs_dssim_cotangents(frame, ptr(image), ptr(target), ptr(image_tangent), nu, lam, gn_floor,
                                int(want_grad), ptr(cot), ptr(loss_out), ptr(workspace),
                                workspace.numel() * workspace.element_size(), ptr(status), stream_handle(stream)),
          "gs_dssim_cotangents")


# ------------------------------------------------------------ batches
def batch_items(items) -> "C.Array":
    """A host array of gs_batch_item from a sequence of them."""
    arr = (gs_batch_item * len(items))()
    for k, it in enumerate(items):
        arr[k] = it
    return arr


def gs_project_batch(items, n_pad_max: int, frame: gs_frame, probe: gs_probe | None, out: gs_projected,
                     status=None, stream=None) -> None:
    L = load()
    arr = batch_items(items)
    check(L.gs_project_batch(arr, len(items), n_pad_max, frame, C.byref(probe) if probe else None, C.byref(out),
                             ptr(status), stream_handle(stream)), "gs_project_batch")


def gs_raster_bwd_batch(items, n_pad_max: int, frame: gs_frame, proj: gs_projected, sorted_: gs_sorted, image,
                        target, final_T, n_contrib, image_tangent, probe: gs_probe | None, loss: gs_loss, loss_out,
                        workspace, status=None, stream=None) -> None:
    L = load()
    arr = batch_items(items)
    check(L.gs_raster_bwd_batch(arr, len(items), n_pad_max, frame, C.byref(proj), C.byref(sorted_), ptr(image),
                                ptr(target), ptr(final_T), ptr(n_contrib), ptr(image_tangent),
                                C.byref(probe) if probe else None, loss, ptr(loss_out), ptr(workspace),
                                workspace.numel() * workspace.element_size(), ptr(status), stream_handle(stream)),
          "gs_raster_bwd_batch")


def gs_tr_update_batch(items, cfg: gs_tr_config, status=None, stream=None) -> None:
    L = load()
    arr = batch_items(items)
    check(L.gs_tr_update_batch(arr, len(items), C.byref(cfg), ptr(status), stream_handle(stream)),
          "gs_tr_update_batch")
