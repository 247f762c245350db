"""Thin ctypes binding of libkfuse.so (include/kfuse.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic
of the chain; all compute runs in the library's CUDA kernels. Device buffers are torch
tensors owned by the caller; streams are torch.cuda streams (default: the current one).
If libkfuse.so has not been built, importing works but the first call raises.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkfuse.so")

KF_OK, KF_EINVAL, KF_ENOMEM, KF_ECUDA, KF_ESMEM, KF_EUNSUPPORTED, KF_ESTATE, KF_ETIMEOUT = range(8)
KF_PREC_F32, KF_PREC_F16, KF_PREC_F16_TILES = 0, 1, 2
KF_DT_U8, KF_DT_F32, KF_DT_F16, KF_DT_U16 = 0, 1, 2, 3
NSTAGES = 8
STAGE_NAMES = ("convert", "gauss_h", "gauss_v", "sobel", "products", "box5", "harris", "nms")
MAP_CHANNELS = (1, 1, 1, 1, 2, 3, 3, 1, 1)  # index = 1-based stage writing the map (0 = frames)


class KfuseError(RuntimeError):
    def __init__(self, call: str, status: int, cuda: int = 0):
        self.status, self.cuda = status, cuda
        msg = f"{call} failed: {_lib().kf_status_str(status).decode()} (status {status})"
        if status == KF_ECUDA:
            msg += f", CUDA error {cuda}"
        super().__init__(msg)


class kf_stage_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rx", ctypes.c_int), ("ry", ctypes.c_int), ("rt", ctypes.c_int),
                ("in_bytes", ctypes.c_double), ("out_bytes", ctypes.c_double)]


class kf_geometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("W", "H", "T", "box_x", "box_y", "box_t")]


class kf_video(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_void_p), ("W", ctypes.c_int64), ("H", ctypes.c_int64),
                ("T", ctypes.c_int64), ("pitch", ctypes.c_int64)]


class kf_corners(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_void_p), ("mask_pitch", ctypes.c_int64), ("counts", ctypes.c_void_p)]


class kf_tracks(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("n_points", ctypes.c_void_p), ("idx", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class kf_map(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p * 3), ("channels", ctypes.c_int), ("dtype", ctypes.c_int),
                ("pitch", ctypes.c_int64), ("frame_stride", ctypes.c_int64)]


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libkfuse.so is not built ({LIB_PATH}); run "
                               "python -m paper_1509_04394_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        sig = {
            "kf_status_str": (ctypes.c_char_p, [i32]),
            "kf_last_cuda_error": (i32, [P]),
            "kf_version": (i32, [P, P]),
            "kf_create": (i32, [i32, P]),
            "kf_destroy": (i32, [P]),
            "kf_device_error": (i32, [P, P]),
            "kf_set_precision": (i32, [P, i32]),
            "kf_set_chunk_rows": (i32, [P, i32]),
            "kf_set_host_chunk_rows": (i32, [P, i32]),
            "kf_set_wait_polls": (i32, [P, ctypes.c_uint32]),
            "kf_add_stage": (i32, [P, P, P]),
            "kf_add_harris_chain": (i32, [P]),
            "kf_num_stages": (i32, [P, P]),
            "kf_group_traffic": (i32, [P, i32, i32, P, P]),
            "kf_group_onchip": (i32, [P, i32, i32, P, P]),
            "kf_partition_traffic": (i32, [P, u32, P, P]),
            "kf_plan": (i32, [P, P, dbl, P, P]),
            "kf_enumerate": (i32, [P, P, i64, P]),
            "kf_map_scale": (i32, [P, i32, P]),
            "kf_workspace_bytes": (i32, [P, u32, i64, i64, i64, P]),
            "kf_run": (i32, [P, u32, P, P, P, ctypes.c_size_t, P]),
            "kf_run_group": (i32, [P, i32, i32, P, P, i64, i64, i64, P, P]),
            "kf_run_static": (i32, [P, u32, P, P, P]),
            "kf_track_workspace_bytes": (i32, [P, i64, i64, i64, P]),
            "kf_track": (i32, [P, P, P, P, P, ctypes.c_size_t, P]),
            "kf_track_host": (i32, [P, P, P, P, P, P, P, P, ctypes.c_size_t, i64, i32, P]),
            "kf_batch_workspace_bytes": (i32, [P, P, i32, i32, P]),
            "kf_batch_create": (i32, [P, P, P, P, i32, P, ctypes.c_size_t, P]),
            "kf_batch_create_ex": (i32, [P, P, P, P, i32, P, i32, P, ctypes.c_size_t, P]),
            "kf_batch_run": (i32, [P, P]),
            "kf_batch_destroy": (i32, [P]),
            "kf_tune_chunk_rows": (i32, [P, P, P, P, i32, i32, P, P, P]),
            "kf_tune_track_rows": (i32, [P, P, P, P, P, ctypes.c_size_t, P, i32, i32, P, P, P]),
            "kf_plan_measured": (i32, [P, P, P, P, ctypes.c_size_t, P, i32, i32, P, P, P, P]),
            "kf_dag_create": (i32, [P, P, i32, P]),
            "kf_dag_destroy": (i32, [P]),
            "kf_dag_group_info": (i32, [P, i32, i32, i64, i64, i64, P, P, P]),
            "kf_dag_plan": (i32, [P, P, P, P]),
            "kf_dag_workspace_bytes": (i32, [P, i64, i64, i64, P]),
            "kf_dag_run": (i32, [P, u32, P, P, i64, P, ctypes.c_size_t, P]),
            "kf_dag_time_groups": (i32, [P, P, P, i64, P, ctypes.c_size_t, i32, P, P]),
            "kf_costmodel_train": (i32, [P, P, P, i32, i32, ctypes.c_float, ctypes.c_uint, P]),
            "kf_costmodel_predict": (i32, [P, P, i32, P]),
            "kf_costmodel_forward": (i32, [P, P, P, i32, P]),
            "kf_costmodel_grad": (i32, [P, P, P, P, i32, P, P]),
            "kf_costmodel_get": (i32, [P, P, P]),
            "kf_costmodel_set": (i32, [P, P, P]),
            "kf_set_kernel_timing": (i32, [P, i32]),
            "kf_pc_traffic": (i32, [P, u32, i64, i64, i64, P]),
            "kf_pc_plan": (i32, [P, i64, i64, i64, P, P]),
            "kf_pc_workspace_bytes": (i32, [P, u32, i64, i64, i64, P]),
            "kf_pc_run": (i32, [P, u32, P, P, P, ctypes.c_size_t, P]),
            "kf_pc_run_group": (i32, [P, i32, i32, P, P, i64, P, i64, P, P, ctypes.c_size_t, P]),
            "kf_pc_group_workspace_bytes": (i32, [P, i32, i32, i64, i64, i64, P]),
            "kf_pc_kalman": (i32, [P, P, i64, i32, P, P, P]),
            "kf_kernel_times": (i32, [P, P, P]),
            "kf_kernel_timeline": (i32, [P, ctypes.c_int64, P, P, P, P]),
            "kf_st_smem_bytes": (i32, [i32, i32, P]),
            "kf_st_traffic": (i32, [i64, i64, i64, i32, i32, i32, P, P]),
            "kf_st_box_eq6": (i32, [dbl, i32, P, P]),
            "kf_st_run": (i32, [P, P, P, i64, P, i32, i32, i32, P]),
            "kf_st_plan_eq6": (i32, [dbl, i32, P, P]),
            "kf_st_tune": (i32, [P, P, P, i64, P, i32, P, i32, i32, P, P, P, P]),
            "kf_dag_xplan_traffic": (i32, [P, u32, u32, i64, i64, i64, P, P]),
            "kf_dag_plan_recompute": (i32, [P, i64, i64, i64, dbl, P, P, P, P]),
            "kf_dag_run_x": (i32, [P, u32, u32, P, P, i64, P, ctypes.c_size_t, P]),
            "kf_dag_time_xgroups": (i32, [P, P, P, i64, P, ctypes.c_size_t, P, i32, i32, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _L = L
    return _L


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding wraps (all declared in kfuse.h)."""
    return ["kf_status_str", "kf_last_cuda_error", "kf_version", "kf_create", "kf_destroy", "kf_device_error",
            "kf_set_precision", "kf_set_chunk_rows", "kf_set_host_chunk_rows", "kf_set_wait_polls", "kf_add_stage",
            "kf_add_harris_chain",
            "kf_num_stages", "kf_group_traffic", "kf_group_onchip", "kf_partition_traffic", "kf_plan",
            "kf_enumerate", "kf_map_scale", "kf_workspace_bytes", "kf_run", "kf_run_group", "kf_run_static",
            "kf_track_workspace_bytes", "kf_track", "kf_batch_workspace_bytes", "kf_batch_create", "kf_batch_create_ex",
            "kf_batch_run", "kf_batch_destroy", "kf_tune_chunk_rows", "kf_tune_track_rows", "kf_plan_measured",
            "kf_dag_create", "kf_dag_destroy",
            "kf_dag_group_info", "kf_dag_plan", "kf_dag_workspace_bytes", "kf_dag_run", "kf_dag_time_groups",
            "kf_costmodel_train", "kf_costmodel_predict", "kf_costmodel_forward", "kf_costmodel_grad", "kf_costmodel_get",
            "kf_costmodel_set", "kf_set_kernel_timing", "kf_kernel_times", "kf_kernel_timeline",
            "kf_pc_traffic", "kf_pc_plan",
            "kf_pc_workspace_bytes", "kf_pc_run", "kf_pc_run_group", "kf_pc_kalman", "kf_pc_group_workspace_bytes",
            "kf_track_host", "kf_st_smem_bytes", "kf_st_traffic", "kf_st_box_eq6", "kf_st_run", "kf_st_plan_eq6", "kf_st_tune",
            "kf_dag_xplan_traffic", "kf_dag_plan_recompute", "kf_dag_run_x", "kf_dag_time_xgroups"]


def _check(call: str, status: int, ctx=None):
    if status != KF_OK:
        cuda = _lib().kf_last_cuda_error(ctx) if ctx else 0
        raise KfuseError(call, status, cuda)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _geom(W, H, T, box=(0, 0, 0)) -> kf_geometry:
    return kf_geometry(int(W), int(H), int(T), int(box[0]), int(box[1]), int(box[2]))


# ------------------------------------------------------------------ entry points
def kf_version() -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check("kf_version", _lib().kf_version(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def kf_create(device: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check("kf_create", _lib().kf_create(int(device), ctypes.byref(h)))
    return h


def kf_destroy(ctx) -> None:
    _check("kf_destroy", _lib().kf_destroy(ctx))


def kf_device_error(ctx) -> int:
    """Synchronise and return (then clear) the context's device error word."""
    c = ctypes.c_int()
    _check("kf_device_error", _lib().kf_device_error(ctx, ctypes.byref(c)), ctx)
    return c.value


def kf_set_precision(ctx, precision: int) -> None:
    _check("kf_set_precision", _lib().kf_set_precision(ctx, int(precision)), ctx)


def kf_set_chunk_rows(ctx, rows: int) -> None:
    _check("kf_set_chunk_rows", _lib().kf_set_chunk_rows(ctx, int(rows)), ctx)


def kf_set_host_chunk_rows(ctx, rows: int) -> None:
    """Tile height of kf_track_host's chunk launches; 0 chooses it per chunk."""
    _check("kf_set_host_chunk_rows", _lib().kf_set_host_chunk_rows(ctx, int(rows)), ctx)


def kf_set_wait_polls(ctx, polls: int) -> None:
    _check("kf_set_wait_polls", _lib().kf_set_wait_polls(ctx, int(polls)), ctx)


def kf_add_stage(ctx, kind: int, rx: int = 0, ry: int = 0, rt: int = 0, in_bytes: float = 0.0,
                 out_bytes: float = 0.0) -> int:
    d = kf_stage_desc(kind, rx, ry, rt, in_bytes, out_bytes)
    i = ctypes.c_int()
    _check("kf_add_stage", _lib().kf_add_stage(ctx, ctypes.byref(d), ctypes.byref(i)), ctx)
    return i.value


def kf_add_harris_chain(ctx) -> None:
    _check("kf_add_harris_chain", _lib().kf_add_harris_chain(ctx), ctx)


def kf_num_stages(ctx) -> int:
    n = ctypes.c_int()
    _check("kf_num_stages", _lib().kf_num_stages(ctx, ctypes.byref(n)), ctx)
    return n.value


def kf_group_traffic(ctx, first: int, last: int, W, H, T, box=(0, 0, 0)) -> float:
    g, b = _geom(W, H, T, box), ctypes.c_double()
    _check("kf_group_traffic", _lib().kf_group_traffic(ctx, first, last, ctypes.byref(g), ctypes.byref(b)), ctx)
    return b.value


def kf_group_onchip(ctx, first: int, last: int, W, H, T, box=(0, 0, 0)) -> float:
    g, b = _geom(W, H, T, box), ctypes.c_double()
    _check("kf_group_onchip", _lib().kf_group_onchip(ctx, first, last, ctypes.byref(g), ctypes.byref(b)), ctx)
    return b.value


def kf_partition_traffic(ctx, cuts: int, W, H, T, box=(0, 0, 0)) -> float:
    g, b = _geom(W, H, T, box), ctypes.c_double()
    _check("kf_partition_traffic", _lib().kf_partition_traffic(ctx, cuts, ctypes.byref(g), ctypes.byref(b)), ctx)
    return b.value


def kf_plan(ctx, W, H, T, box=(0, 0, 0), onchip_limit: float = math.inf) -> tuple[int, float]:
    g, c, b = _geom(W, H, T, box), ctypes.c_uint32(), ctypes.c_double()
    lim = 1e300 if math.isinf(onchip_limit) else float(onchip_limit)
    _check("kf_plan", _lib().kf_plan(ctx, ctypes.byref(g), lim, ctypes.byref(c), ctypes.byref(b)), ctx)
    return c.value, b.value


def kf_enumerate(ctx) -> list[int]:
    n = ctypes.c_int64()
    _check("kf_enumerate", _lib().kf_enumerate(ctx, None, 0, ctypes.byref(n)), ctx)
    buf = (ctypes.c_uint32 * n.value)()
    _check("kf_enumerate", _lib().kf_enumerate(ctx, buf, n.value, ctypes.byref(n)), ctx)
    return list(buf)


def kf_map_scale(ctx, stage: int) -> float:
    f = ctypes.c_double()
    _check("kf_map_scale", _lib().kf_map_scale(ctx, stage, ctypes.byref(f)), ctx)
    return f.value


def kf_workspace_bytes(ctx, cuts: int, W, H, T) -> int:
    b = ctypes.c_size_t()
    _check("kf_workspace_bytes", _lib().kf_workspace_bytes(ctx, cuts, W, H, T, ctypes.byref(b)), ctx)
    return b.value


def kf_run(ctx, cuts: int, frames, W: int, mask, counts, workspace=None, stream=None) -> None:
    """frames, mask: uint8 CUDA tensors [T, H, pitch]; counts: int32 CUDA tensor [T]."""
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("kf_run", _lib().kf_run(ctx, cuts, ctypes.byref(v), ctypes.byref(o), _ptr(workspace), ws_bytes,
                                   _stream(stream)), ctx)


def kf_track_workspace_bytes(ctx, W, H, T) -> int:
    b = ctypes.c_size_t()
    _check("kf_track_workspace_bytes", _lib().kf_track_workspace_bytes(ctx, W, H, T, ctypes.byref(b)), ctx)
    return b.value


def kf_track(ctx, frames, W: int, mask, counts, K: int, n_points, idx, u, v, status, workspace, stream=None) -> None:
    """Fused chain + corner selection + LK tracking. idx, u, v, status: [T, K] CUDA tensors
    (int32, float32, float32, int32); n_points: int32 [T]."""
    T, H, P = frames.shape
    vid = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    tr = kf_tracks(int(K), n_points.data_ptr(), idx.data_ptr(), u.data_ptr(), v.data_ptr(), status.data_ptr())
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("kf_track", _lib().kf_track(ctx, ctypes.byref(vid), ctypes.byref(o), ctypes.byref(tr), workspace.data_ptr(),
                                       ws_bytes, _stream(stream)), ctx)


KF_MASK_BYTES, KF_MASK_BITS = 0, 1


def kf_track_host(ctx, host, dev, W: int, K: int, workspace, chunk: int = 100, stream=None,
                  mask_format: int = KF_MASK_BYTES) -> None:
    """kf_track from host tensors to host tensors, pipelined in chunks of `chunk` frames
    (copies in, chains on three streams, masks copied out after each chunk's chain,
    tracking of the first half of the frames while later copies arrive). host, dev: dicts of tensors (host: pinned CPU, dev: CUDA) with keys frames [T, H, P]
    u8, mask [T, H, MP] u8 (KF_MASK_BITS: host mask [T, S] u8, S >= ceil(W H / 8) a
    multiple of 16), counts [T] i32, n_points [T] i32, idx / status [T, K] i32, u / v
    [T, K] f32."""
    def structs(d, packed=False):
        T, H, P = d["frames"].shape
        vid = kf_video(d["frames"].data_ptr(), int(W), int(H), int(T), int(P))
        mp = int(d["mask"].shape[1]) if packed else int(d["mask"].shape[2])
        o = kf_corners(d["mask"].data_ptr(), mp, d["counts"].data_ptr())
        tr = kf_tracks(int(K), d["n_points"].data_ptr(), d["idx"].data_ptr(), d["u"].data_ptr(), d["v"].data_ptr(),
                       d["status"].data_ptr())
        return vid, o, tr
    hv, ho, ht = structs(host, mask_format == KF_MASK_BITS)
    dv, do, dt = structs(dev)
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("kf_track_host", _lib().kf_track_host(ctx, ctypes.byref(hv), ctypes.byref(ho), ctypes.byref(ht),
                                                 ctypes.byref(dv), ctypes.byref(do), ctypes.byref(dt),
                                                 workspace.data_ptr(), ws_bytes, int(chunk), int(mask_format),
                                                 _stream(stream)), ctx)


def _videos(frames_list, W_list):
    arr = (kf_video * len(frames_list))()
    for i, (f, W) in enumerate(zip(frames_list, W_list)):
        T, H, P = f.shape
        arr[i] = kf_video(f.data_ptr(), int(W), int(H), int(T), int(P))
    return arr


def kf_batch_workspace_bytes(ctx, frames_list, W_list, K: int = 0) -> int:
    v = _videos(frames_list, W_list)
    b = ctypes.c_size_t()
    _check("kf_batch_workspace_bytes", _lib().kf_batch_workspace_bytes(ctx, v, len(frames_list), int(K), ctypes.byref(b)),
           ctx)
    return b.value


def kf_batch_create(ctx, frames_list, W_list, masks, counts_list, workspace, tracks=None, chunk_rows=None,
                    warps_per_sm: int = 0):
    """tracks: None or a list of (K, n_points, idx, u, v, status) tensors per video;
    chunk_rows: None (the context's) or one tile height per video; warps_per_sm: 0 = as
    many resident warps as fit (kf_batch_create_ex)."""
    n = len(frames_list)
    v = _videos(frames_list, W_list)
    o = (kf_corners * n)(*[kf_corners(m.data_ptr(), int(m.shape[2]), c.data_ptr()) for m, c in zip(masks, counts_list)])
    tr = None
    if tracks is not None:
        tr = (kf_tracks * n)(*[kf_tracks(int(K), a.data_ptr(), b.data_ptr(), c.data_ptr(), d.data_ptr(), e.data_ptr())
                               for (K, a, b, c, d, e) in tracks])
    h = ctypes.c_void_p()
    ws_bytes = workspace.numel() * workspace.element_size()
    rows = None if chunk_rows is None else (ctypes.c_int * n)(*[int(r) for r in chunk_rows])
    _check("kf_batch_create_ex", _lib().kf_batch_create_ex(ctx, v, o, tr, n, rows, int(warps_per_sm), workspace.data_ptr(),
                                                           ws_bytes, ctypes.byref(h)), ctx)
    return h


def kf_batch_run(batch, stream=None) -> None:
    _check("kf_batch_run", _lib().kf_batch_run(batch, _stream(stream)))


def kf_batch_destroy(batch) -> None:
    _check("kf_batch_destroy", _lib().kf_batch_destroy(batch))


def kf_tune_chunk_rows(ctx, frames, W: int, mask, counts, candidates, reps: int = 3, stream=None):
    T, H, P = frames.shape
    vid = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    cand = (ctypes.c_int * len(candidates))(*candidates)
    best, ms = ctypes.c_int(), ctypes.c_float()
    _check("kf_tune_chunk_rows", _lib().kf_tune_chunk_rows(ctx, ctypes.byref(vid), ctypes.byref(o), cand, len(candidates),
                                                           int(reps), _stream(stream), ctypes.byref(best),
                                                           ctypes.byref(ms)), ctx)
    return best.value, ms.value


def kf_tune_track_rows(ctx, frames, W: int, mask, counts, K: int, n_points, idx, u, v, status, workspace, candidates,
                       reps: int = 3, stream=None):
    """The tile-height autotuner on kf_track (same tensors); returns (best rows, its ms)."""
    T, H, P = frames.shape
    vid = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    tr = kf_tracks(int(K), n_points.data_ptr(), idx.data_ptr(), u.data_ptr(), v.data_ptr(), status.data_ptr())
    cand = (ctypes.c_int * len(candidates))(*candidates)
    best, ms = ctypes.c_int(), ctypes.c_float()
    _check("kf_tune_track_rows", _lib().kf_tune_track_rows(
        ctx, ctypes.byref(vid), ctypes.byref(o), ctypes.byref(tr), workspace.data_ptr(),
        workspace.numel() * workspace.element_size(), cand, len(candidates), int(reps), _stream(stream),
        ctypes.byref(best), ctypes.byref(ms)), ctx)
    return best.value, ms.value


def kf_plan_measured(ctx, frames, W: int, mask, counts, workspace, candidates=None, reps: int = 3, stream=None):
    """Measured exhaustive partition choice: (best cut mask, its median ms, every candidate's
    median ms in candidate order). candidates=None times all 2^(n-1) partitions."""
    import numpy as np
    T, H, P = frames.shape
    vid = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    n = len(candidates) if candidates is not None else 1 << 7
    cand = (ctypes.c_uint32 * n)(*candidates) if candidates is not None else None
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    best, ms = ctypes.c_uint32(), ctypes.c_float()
    all_ms = np.zeros(n, dtype=np.float32)
    _check("kf_plan_measured", _lib().kf_plan_measured(ctx, ctypes.byref(vid), ctypes.byref(o), _ptr(workspace), ws_bytes,
                                                       cand, n if candidates is not None else 0, int(reps),
                                                       _stream(stream), ctypes.byref(best), ctypes.byref(ms),
                                                       all_ms.ctypes.data), ctx)
    return best.value, ms.value, all_ms


KF_NFEAT = 12


class kf_gstage(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("in1", ctypes.c_int), ("in2", ctypes.c_int), ("radius", ctypes.c_int),
                ("a", ctypes.c_float), ("b", ctypes.c_float)]


def kf_dag_create(ctx, rows):
    """rows: (kind, in1, in2, radius, a, b) per stage (synth.dags.to_array)."""
    arr = (kf_gstage * len(rows))(*[kf_gstage(int(k), int(i1), int(i2), int(r), float(a), float(b))
                                    for (k, i1, i2, r, a, b) in rows])
    h = ctypes.c_void_p()
    _check("kf_dag_create", _lib().kf_dag_create(ctx, arr, len(rows), ctypes.byref(h)), ctx)
    return h


def kf_dag_destroy(dag) -> None:
    _check("kf_dag_destroy", _lib().kf_dag_destroy(dag))


def kf_dag_group_info(dag, first: int, last: int, W, H, T):
    """(features [KF_NFEAT], on-chip bytes, traffic bytes) of group [first, last]."""
    f = (ctypes.c_float * KF_NFEAT)()
    oc_, tr = ctypes.c_double(), ctypes.c_double()
    _check("kf_dag_group_info", _lib().kf_dag_group_info(dag, first, last, W, H, T, f, ctypes.byref(oc_),
                                                         ctypes.byref(tr)))
    return list(f), oc_.value, tr.value


def kf_dag_plan(dag, group_cost) -> tuple[int, float]:
    arr = (ctypes.c_double * len(group_cost))(*[float(c) for c in group_cost])
    c, cost = ctypes.c_uint32(), ctypes.c_double()
    _check("kf_dag_plan", _lib().kf_dag_plan(dag, arr, ctypes.byref(c), ctypes.byref(cost)))
    return c.value, cost.value


def kf_dag_workspace_bytes(dag, W, H, T) -> int:
    b = ctypes.c_size_t()
    _check("kf_dag_workspace_bytes", _lib().kf_dag_workspace_bytes(dag, W, H, T, ctypes.byref(b)))
    return b.value


def kf_dag_run(dag, cuts: int, frames, W: int, out, workspace, stream=None) -> None:
    """frames: uint8 [T, H, pitch]; out: float32 [T, H, opitch] (CUDA tensors)."""
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    _check("kf_dag_run", _lib().kf_dag_run(dag, cuts, ctypes.byref(v), out.data_ptr(), int(out.shape[2]),
                                           workspace.data_ptr(), workspace.numel(), _stream(stream)))


def kf_dag_xplan_traffic(dag, cuts: int, inline_mask: int, W, H, T) -> tuple[float, float]:
    """(traffic bytes, largest on-chip bytes per block) of plan (cuts, inline_mask)."""
    b, m = ctypes.c_double(), ctypes.c_double()
    _check("kf_dag_xplan_traffic", _lib().kf_dag_xplan_traffic(dag, int(cuts), int(inline_mask), int(W), int(H), int(T),
                                                               ctypes.byref(b), ctypes.byref(m)))
    return b.value, m.value


def kf_dag_plan_recompute(dag, W, H, T, onchip_limit: float = 0.0, model=None) -> tuple[int, int, float]:
    """(cuts, inline_mask, cost) of the cheapest plan: cost = traffic bytes, or the
    learned model's predicted ms when `model` (a context with a trained model) is given."""
    c, x, b = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
    _check("kf_dag_plan_recompute", _lib().kf_dag_plan_recompute(dag, int(W), int(H), int(T), float(onchip_limit), model,
                                                                 ctypes.byref(c), ctypes.byref(x), ctypes.byref(b)))
    return c.value, x.value, b.value


def kf_dag_run_x(dag, cuts: int, inline_mask: int, frames, W: int, out, workspace, stream=None) -> None:
    """kf_dag_run with inlined (recomputed) nodes."""
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    _check("kf_dag_run_x", _lib().kf_dag_run_x(dag, int(cuts), int(inline_mask), ctypes.byref(v), out.data_ptr(),
                                               int(out.shape[2]), workspace.data_ptr(), workspace.numel(),
                                               _stream(stream)))


def kf_dag_time_xgroups(dag, groups, frames, W: int, out, workspace, reps: int = 2, stream=None):
    """groups: [(first, last, inline_mask)] -> (ms [G], features [G, KF_NFEAT])."""
    import numpy as np
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    g = np.ascontiguousarray(np.array(groups, dtype=np.int32).reshape(-1, 3))
    G = g.shape[0]
    ms = np.zeros(G, dtype=np.float32)
    feats = np.zeros((G, KF_NFEAT), dtype=np.float32)
    _check("kf_dag_time_xgroups", _lib().kf_dag_time_xgroups(dag, ctypes.byref(v), out.data_ptr(), int(out.shape[2]),
                                                             workspace.data_ptr(), workspace.numel(),
                                                             g.ctypes.data, int(G), int(reps), _stream(stream),
                                                             ms.ctypes.data, feats.ctypes.data))
    return ms, feats


def group_index(n: int, a: int, b: int) -> int:
    """Index of 0-based group [a, b] among the n(n+1)/2 candidate groups."""
    return a * n - a * (a - 1) // 2 + (b - a)


def kf_dag_time_groups(dag, n: int, frames, W: int, out, workspace, reps: int = 3, stream=None) -> list[float]:
    """Measured mean time (ms) of every candidate group of an n-stage DAG, -1 if infeasible."""
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    ms = (ctypes.c_float * (n * (n + 1) // 2))()
    _check("kf_dag_time_groups", _lib().kf_dag_time_groups(dag, ctypes.byref(v), out.data_ptr(), int(out.shape[2]),
                                                           workspace.data_ptr(), workspace.numel(), int(reps),
                                                           _stream(stream), ms))
    return list(ms)


KF_MLP_NPARAMS = 64 * KF_NFEAT + 64 + 64 * 64 + 64 + 64 + 1


def _fptr(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data


def kf_costmodel_train(ctx, features, ms, steps: int = 2000, lr: float = 3e-3, seed: int = 0) -> float:
    """features: [n, KF_NFEAT], ms: [n] (numpy). Returns the final standardised MSE."""
    f, fp = _fptr(features)
    m, mp = _fptr(ms)
    loss = ctypes.c_float()
    _check("kf_costmodel_train", _lib().kf_costmodel_train(ctx, fp, mp, int(m.shape[0]), int(steps), float(lr),
                                                           int(seed), ctypes.byref(loss)), ctx)
    return loss.value


def kf_costmodel_predict(ctx, features):
    import numpy as np
    f, fp = _fptr(features)
    out = np.empty(f.shape[0], dtype=np.float32)
    _check("kf_costmodel_predict", _lib().kf_costmodel_predict(ctx, fp, int(f.shape[0]), out.ctypes.data), ctx)
    return out


def kf_costmodel_forward(ctx, params, x):
    """The raw network at `params` for the rows of x, on the context's GPU."""
    import numpy as np
    p, pp = _fptr(params)
    xx, xp = _fptr(x)
    out = np.empty(xx.shape[0], dtype=np.float32)
    _check("kf_costmodel_forward", _lib().kf_costmodel_forward(ctx, pp, xp, int(xx.shape[0]), out.ctypes.data), ctx)
    return out


def kf_costmodel_grad(ctx, params, x, y):
    import numpy as np
    p, pp = _fptr(params)
    xx, xp = _fptr(x)
    yy, yp = _fptr(y)
    g = np.empty(KF_MLP_NPARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check("kf_costmodel_grad", _lib().kf_costmodel_grad(ctx, pp, xp, yp, int(yy.shape[0]), g.ctypes.data,
                                                         ctypes.byref(loss)), ctx)
    return loss.value, g


def kf_costmodel_get(ctx):
    import numpy as np
    p = np.empty(KF_MLP_NPARAMS, dtype=np.float32)
    nrm = np.empty(2 * KF_NFEAT + 2, dtype=np.float32)
    _check("kf_costmodel_get", _lib().kf_costmodel_get(ctx, p.ctypes.data, nrm.ctypes.data), ctx)
    return p, nrm


def kf_costmodel_set(ctx, params, norm) -> None:
    p, pp = _fptr(params)
    n, np_ = _fptr(norm)
    _check("kf_costmodel_set", _lib().kf_costmodel_set(ctx, pp, np_), ctx)


KF_STATIC_WORKSPACE_BYTES = 64 << 20


def kf_run_static(ctx, cuts: int, frames, W: int, mask, counts, stream=None) -> None:
    """kf_run with the library's fixed per-GPU workspace: for callers that cannot allocate
    device memory. Same tensors as kf_run, no workspace argument."""
    T, H, P = frames.shape
    v = kf_video(frames.data_ptr(), int(W), int(H), int(T), int(P))
    o = kf_corners(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr())
    _check("kf_run_static", _lib().kf_run_static(ctx, cuts, ctypes.byref(v), ctypes.byref(o), _stream(stream)), ctx)


KF_KT_GROUP, KF_KT_CHAIN_CORNERS, KF_KT_SELECT, KF_KT_LK = 0, 1, 2, 3
KF_KT_PACK, KF_KT_COPY_IN, KF_KT_COPY_OUT, KF_KT_COUNT = 4, 5, 6, 7
KERNEL_KINDS = ("group", "chain_corners", "select", "lk", "pack", "copy_in", "copy_out")


def kf_set_kernel_timing(ctx, on: bool) -> None:
    """Bracket every kernel the context launches with CUDA events on its stream."""
    _check("kf_set_kernel_timing", _lib().kf_set_kernel_timing(ctx, 1 if on else 0), ctx)


def kf_kernel_times(ctx) -> dict[str, tuple[int, float]]:
    """Per kernel kind: (launches, summed ms) since the previous call; clears the record."""
    n = (ctypes.c_int64 * KF_KT_COUNT)()
    ms = (ctypes.c_double * KF_KT_COUNT)()
    _check("kf_kernel_times", _lib().kf_kernel_times(ctx, n, ms), ctx)
    return {KERNEL_KINDS[k]: (int(n[k]), float(ms[k])) for k in range(KF_KT_COUNT)}


def kf_kernel_timeline(ctx, cap: int = 4096) -> list[tuple[str, float, float]]:
    """The recorded launches and copies in enqueue order: (kind, start ms, end ms) from the
    earliest start; clears the record."""
    n = ctypes.c_int64()
    kinds = (ctypes.c_int * cap)()
    t0 = (ctypes.c_double * cap)()
    t1 = (ctypes.c_double * cap)()
    _check("kf_kernel_timeline", _lib().kf_kernel_timeline(ctx, cap, ctypes.byref(n), kinds, t0, t1), ctx)
    return [(KERNEL_KINDS[kinds[i]], float(t0[i]), float(t1[i])) for i in range(min(n.value, cap))]


def make_map(planes, dtype: int) -> kf_map:
    """kf_map over a list of CUDA tensors [T, H, pitch] (one per channel)."""
    m = kf_map()
    for i, t in enumerate(planes):
        m.plane[i] = t.data_ptr()
    m.channels = len(planes)
    m.dtype = dtype
    m.pitch = int(planes[0].shape[2])
    m.frame_stride = int(planes[0].shape[1] * planes[0].shape[2])
    return m


def kf_run_group(ctx, first: int, last: int, in_planes, in_dtype: int, out_planes, out_dtype: int, W: int,
                 counts=None, stream=None) -> None:
    """Run fused group [first, last] (0-based) from map planes to map planes."""
    T, H, _ = in_planes[0].shape
    mi, mo = make_map(in_planes, in_dtype), make_map(out_planes, out_dtype)
    _check("kf_run_group", _lib().kf_run_group(ctx, first, last, ctypes.byref(mi), ctypes.byref(mo), int(W), int(H),
                                               int(T), _ptr(counts), _stream(stream)), ctx)


# ------------------------------------------------------------------ convenience
class Context:
    """Owns one kf_ctx; the methods are the entry points above with the handle bound."""

    def __init__(self, device: int = 0, precision: int = KF_PREC_F32, harris: bool = True):
        self.h = kf_create(device)
        self.device = device
        if precision != KF_PREC_F32:
            kf_set_precision(self.h, precision)
        self.precision = precision
        if harris:
            kf_add_harris_chain(self.h)

    def close(self):
        if self.h:
            kf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __getattr__(self, name):
        f = globals().get("kf_" + name)
        if f is None:
            raise AttributeError(name)
        return lambda *a, **k: f(self.h, *a, **k)


# ------------------------------------------------------------------ the paper's own chain
KF_PC_STAGES, KF_PC_REGIONS = 5, 16
PC_SCALE = (65280.0, 65280.0, 16 * 65280.0, 16 * 65280.0)  # stage maps 0..3: scaled = true * scale


class kf_pc_video(ctypes.Structure):
    _fields_ = [("rgba", ctypes.c_void_p), ("W", ctypes.c_int64), ("H", ctypes.c_int64), ("T", ctypes.c_int64),
                ("pitch", ctypes.c_int64)]


class kf_pc_out(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_void_p), ("mask_pitch", ctypes.c_int64), ("counts", ctypes.c_void_p),
                ("regions", ctypes.c_void_p)]


def _pc_video(frames, W: int, T: int | None = None, H: int | None = None):
    """frames: uint8 tensor [T, H, pitch, 4] (RGBA), or None with explicit T and H."""
    if frames is None:
        return kf_pc_video(0, int(W), int(H), int(T), int(W))
    t, h, pitch, c = frames.shape
    assert c == 4
    return kf_pc_video(frames.data_ptr(), int(W), int(h), int(t), int(pitch))


def _pc_out(mask, counts, regions):
    return kf_pc_out(mask.data_ptr(), int(mask.shape[2]), counts.data_ptr(), regions.data_ptr())


def kf_pc_traffic(ctx, cuts: int, W: int, H: int, T: int) -> float:
    b = ctypes.c_double()
    _check("kf_pc_traffic", _lib().kf_pc_traffic(ctx, int(cuts), int(W), int(H), int(T), ctypes.byref(b)), ctx)
    return b.value


def kf_pc_plan(ctx, W: int, H: int, T: int) -> tuple[int, float]:
    c, b = ctypes.c_uint32(), ctypes.c_double()
    _check("kf_pc_plan", _lib().kf_pc_plan(ctx, int(W), int(H), int(T), ctypes.byref(c), ctypes.byref(b)), ctx)
    return c.value, b.value


def kf_pc_workspace_bytes(ctx, cuts: int, W: int, H: int, T: int) -> int:
    n = ctypes.c_size_t()
    _check("kf_pc_workspace_bytes", _lib().kf_pc_workspace_bytes(ctx, int(cuts), int(W), int(H), int(T),
                                                                   ctypes.byref(n)), ctx)
    return n.value


def kf_pc_run(ctx, cuts: int, frames, W: int, mask, counts, regions, workspace=None, stream=None) -> None:
    """frames [T, H, pitch, 4] u8 RGBA; mask [T, H, mask_pitch] u8; counts [T] int32;
    regions [T, 16, 3] int32 (all CUDA tensors)."""
    v = _pc_video(frames, W)
    o = _pc_out(mask, counts, regions)
    ws = 0 if workspace is None else workspace.data_ptr()
    nb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("kf_pc_run", _lib().kf_pc_run(ctx, int(cuts), ctypes.byref(v), ctypes.byref(o), ws, nb, _stream(stream)),
           ctx)


def kf_pc_group_workspace_bytes(ctx, a: int, b: int, W: int, H: int, T: int) -> int:
    n = ctypes.c_size_t()
    _check("kf_pc_group_workspace_bytes", _lib().kf_pc_group_workspace_bytes(ctx, int(a), int(b), int(W), int(H), int(T),
                                                                               ctypes.byref(n)), ctx)
    return n.value


def kf_pc_run_group(ctx, a: int, b: int, W: int, frames=None, inp=None, out=None, mask_out=None, workspace=None,
                    stream=None) -> None:
    """One group [a..b]: input RGBA frames (a == 0) or an FP32 map [T, H, pitch]; output an
    FP32 map [T, H, pitch] (b < 4) or (mask, counts, regions) (b == 4). A group holding the
    IIR filter (a <= 1 <= b) needs `workspace` (kf_pc_group_workspace_bytes)."""
    if frames is not None:
        v = _pc_video(frames, W)
    else:
        v = kf_pc_video(0, int(W), int(inp.shape[1]), int(inp.shape[0]), int(W))
    ip = 0 if inp is None else inp.data_ptr()
    ipitch = 0 if inp is None else int(inp.shape[2])
    op_ = 0 if out is None else out.data_ptr()
    opitch = 0 if out is None else int(out.shape[2])
    mo = None if mask_out is None else _pc_out(*mask_out)
    ws = 0 if workspace is None else workspace.data_ptr()
    nb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("kf_pc_run_group", _lib().kf_pc_run_group(ctx, int(a), int(b), ctypes.byref(v), ip, ipitch, op_, opitch,
                                                       ctypes.byref(mo) if mo is not None else None, ws, nb,
                                                       _stream(stream)), ctx)


def kf_pc_kalman(ctx, regions, states, status, stream=None) -> None:
    """regions [T, N, 3] int32 -> states [T, N, 4] float64, status [T, N] int32 (CUDA tensors)."""
    T, N, _ = regions.shape
    _check("kf_pc_kalman", _lib().kf_pc_kalman(ctx, regions.data_ptr(), int(T), int(N), states.data_ptr(),
                                               status.data_ptr(), _stream(stream)), ctx)


# ---------------------------------------------------------------- spatio-temporal boxes
ST_TAPS = (1, 2, 4)


def kf_st_smem_bytes(n: int, x: int) -> int:
    b = ctypes.c_size_t()
    _check("kf_st_smem_bytes", _lib().kf_st_smem_bytes(int(n), int(x), ctypes.byref(b)))
    return b.value


def kf_st_traffic(W: int, H: int, T: int, x: int, t: int, n: int) -> tuple[float, float]:
    """(model bytes, clipped bytes) of the box tiling."""
    m, c = ctypes.c_double(), ctypes.c_double()
    _check("kf_st_traffic", _lib().kf_st_traffic(int(W), int(H), int(T), int(x), int(t), int(n), ctypes.byref(m),
                                                 ctypes.byref(c)))
    return m.value, c.value


def kf_st_box_eq6(beta: float, n: int) -> tuple[float, float]:
    x, t = ctypes.c_double(), ctypes.c_double()
    _check("kf_st_box_eq6", _lib().kf_st_box_eq6(float(beta), int(n), ctypes.byref(x), ctypes.byref(t)))
    return x.value, t.value


def kf_st_run(ctx, frames, W: int, mask, counts, n: int, x: int, t: int, stream=None) -> None:
    """frames [T, H, pitch, 4] u8 RGBA; mask [T, H, mask_pitch] u8; counts [T] int32 (CUDA)."""
    v = _pc_video(frames, W)
    _check("kf_st_run", _lib().kf_st_run(ctx, ctypes.byref(v), mask.data_ptr(), int(mask.shape[2]), counts.data_ptr(),
                                         int(n), int(x), int(t), _stream(stream)), ctx)


def kf_st_plan_eq6(beta: float, n: int) -> tuple[int, int]:
    """The supported box (x, t) nearest Eq. 6 for output volume beta."""
    x, t = ctypes.c_int(), ctypes.c_int()
    _check("kf_st_plan_eq6", _lib().kf_st_plan_eq6(float(beta), int(n), ctypes.byref(x), ctypes.byref(t)))
    return x.value, t.value


def kf_st_tune(ctx, frames, W: int, mask, counts, n: int, boxes, reps: int = 3, stream=None) -> tuple[int, int, float]:
    """The fastest of the candidate boxes [(x, t), ...] on this video: (x, t, ms)."""
    v = _pc_video(frames, W)
    arr = (ctypes.c_int * (2 * len(boxes)))(*[int(a) for xt in boxes for a in xt])
    bx, bt, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check("kf_st_tune", _lib().kf_st_tune(ctx, ctypes.byref(v), mask.data_ptr(), int(mask.shape[2]), counts.data_ptr(),
                                           int(n), arr, len(boxes), int(reps), _stream(stream), ctypes.byref(bx),
                                           ctypes.byref(bt), ctypes.byref(ms)), ctx)
    return bx.value, bt.value, ms.value
