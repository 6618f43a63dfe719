"""Thin ctypes binding of librecon (include/recon.h).

Functions keep the C names and only marshal arguments: numpy arrays (host),
torch tensors (host or CUDA) or raw integer addresses become pointers, the
C structs are mirrored field by field, and a non-zero status raises
ReconError with the library's message.  Every step of the computation runs
inside librecon's CUDA kernels; there is no Python or CPU fallback, and a
missing or unbuildable library raises.
"""
import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

RECON_OK, RECON_EINVAL, RECON_ENOMEM, RECON_ECUDA, RECON_ETIMEOUT, RECON_ESTATE = range(6)
STATUS_NAMES = {0: "RECON_OK", 1: "RECON_EINVAL", 2: "RECON_ENOMEM", 3: "RECON_ECUDA", 4: "RECON_ETIMEOUT",
                5: "RECON_ESTATE"}
RECON_EV_F32_SOA, RECON_EV_PACKED_I16_F16 = 0, 1


class ReconError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class recon_geometry(C.Structure):
    _fields_ = [("radius_mm", C.c_double), ("axial_len_mm", C.c_double), ("max_axial_angle_deg", C.c_double)]


class recon_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("vx", C.c_double), ("vy", C.c_double), ("vz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class recon_events(C.Structure):
    _fields_ = [("fmt", C.c_int32), ("on_device", C.c_int32), ("n", C.c_int64), ("planes", C.c_void_p * 7),
                ("lattice_mm", C.c_double), ("weight", C.c_void_p)]


class recon_region(C.Structure):
    _fields_ = [("z_lo", C.c_int32), ("z_hi", C.c_int32)]


class recon_launch(C.Structure):
    _fields_ = [("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk_events", C.c_int32),
                ("cached_pieces", C.c_int32), ("tail_eval", C.c_int32), ("reduction", C.c_int32),
                ("image_tiling", C.c_int32), ("lanes_per_event", C.c_int32)]


class recon_info(C.Structure):
    _fields_ = [("sigma_mm", C.c_double), ("k_sigma", C.c_double), ("n_vox", C.c_int64),
                ("n_events_resident", C.c_int64), ("has_sensitivity", C.c_int32), ("num_sms", C.c_int32),
                ("sens_total", C.c_double), ("tile_cells", C.c_int64), ("tile_events", C.c_int64),
                ("tile_fallback_events", C.c_int64), ("tile_cell_voxels", C.c_int32), ("tile_halo", C.c_int32 * 3),
                ("subsets", C.c_int32), ("lut_samples", C.c_int32), ("device_bytes", C.c_int64)]


class recon_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("pass_launches", C.c_int64), ("pass_ms", C.c_double),
                ("update_ms", C.c_double), ("autotune_runs", C.c_int64)]


# every extern "C" entry point of include/recon.h with its ctypes signature
_CTX = C.c_void_p
_VP = C.c_void_p
SIGNATURES = {
    "recon_create": (C.c_int, [C.POINTER(recon_geometry), C.POINTER(recon_grid), C.c_double, C.POINTER(C.c_void_p)]),
    "recon_destroy": (None, [_CTX]),
    "recon_last_error": (C.c_char_p, [_CTX]),
    "recon_set_stream": (C.c_int, [_CTX, _VP]),
    "recon_set_kernel_window": (C.c_int, [_CTX, C.c_double]),
    "recon_set_gather_bf16": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_brick_layout": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_projector": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "recon_set_median_filter": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_subsets": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_start_image": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_tiled_pass": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "recon_set_event_order": (C.c_int, [_CTX, C.c_int32, C.c_int32, C.c_int32]),
    "recon_preprocess": (C.c_int, [_CTX, C.POINTER(recon_events), _VP, C.c_double, C.c_int32, _VP, _VP,
                                   C.POINTER(C.c_int64)]),
    "recon_median_filter": (C.c_int, [_CTX, _VP, _VP]),
    "recon_get_tof_samples": (C.c_int, [_CTX, C.c_int32, _VP, _VP, C.POINTER(C.c_int32)]),
    "recon_set_launch": (C.c_int, [_CTX, C.POINTER(recon_launch)]),
    "recon_get_launch": (C.c_int, [_CTX, C.POINTER(recon_launch)]),
    "recon_set_timing": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_graphs": (C.c_int, [_CTX, C.c_int32]),
    "recon_set_autotune": (C.c_int, [_CTX, C.c_int32]),
    "recon_get_info": (C.c_int, [_CTX, C.POINTER(recon_info)]),
    "recon_get_stats": (C.c_int, [_CTX, C.POINTER(recon_stats)]),
    "recon_reset_stats": (C.c_int, [_CTX]),
    "recon_sensitivity": (C.c_int, [_CTX, _VP, C.c_int64, C.c_int32, _VP]),
    "recon_set_sensitivity": (C.c_int, [_CTX, _VP, C.c_int32]),
    "recon_load_events": (C.c_int, [_CTX, C.POINTER(recon_events)]),
    "recon_forward": (C.c_int, [_CTX, C.POINTER(recon_events), _VP, _VP]),
    "recon_backproject": (C.c_int, [_CTX, C.POINTER(recon_events), _VP, _VP]),
    "recon_mlem": (C.c_int, [_CTX, C.POINTER(recon_events), C.c_int32, _VP, _VP, _VP]),
    "recon_event_pass": (C.c_int, [_CTX, C.POINTER(recon_events), _VP, C.c_int32, _VP, C.POINTER(C.c_double)]),
    "recon_update": (C.c_int, [_CTX, _VP, _VP, C.POINTER(C.c_double)]),
    "recon_split_regions": (C.c_int, [_CTX, C.POINTER(recon_events), C.c_int32, C.POINTER(recon_region),
                                      C.c_double, C.c_double, _VP, _VP, _VP]),
    "recon_mlem_regions": (C.c_int, [_CTX, C.POINTER(recon_events), C.c_int32, C.POINTER(recon_region),
                                     C.c_double, C.c_double, C.c_int32, _VP, _VP, _VP]),
    "recon_set_region_block": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "recon_region_slab_voxels": (C.c_int, [_CTX, C.c_int32, C.POINTER(recon_region), C.c_double,
                                           C.POINTER(C.c_int64)]),
    "recon_debug_fail_alloc": (C.c_int, [C.c_int64]),
    "recon_debug_bounds_violations": (C.c_int, [C.POINTER(C.c_int64)]),
    "recon_split_regions_noalloc": (C.c_int, [C.POINTER(recon_grid), C.POINTER(recon_events), C.c_int32,
                                              C.POINTER(recon_region), C.c_double, _VP, _VP, _VP, C.c_int64, _VP]),
}

_lib = None
_lock = threading.Lock()


def library_path():
    """librecon.so, or with RECON_BOUNDS_CHECK=1 in the environment the bounds-checked
    build librecon_check.so."""
    return _build.CHECK_LIB if os.environ.get("RECON_BOUNDS_CHECK") == "1" else _build.LIB


def load():
    """Load the library (library_path()), building it first when a source is newer."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            checked = path == _build.CHECK_LIB
            if not _build.up_to_date(path):
                try:
                    _build.build(checked=checked)
                except Exception as e:  # no CPU fallback: the CUDA library is the only path
                    raise ReconError(RECON_ECUDA, f"{os.path.basename(path)} is missing and could not be built: "
                                                  f"{e}") from e
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def ptr(x):
    """Address of a numpy array, torch tensor or raw int (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if getattr(x, "is_cuda", False):
            # the library orders its work only after its own stream: torch work still
            # queued on another stream that writes or reads this tensor must finish first
            import torch
            torch.cuda.current_stream(x.device).synchronize()
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _on_device(x):
    return bool(getattr(x, "is_cuda", False))


def check(ctx, status):
    if status != RECON_OK:
        msg = load().recon_last_error(ctx)
        raise ReconError(status, msg.decode() if msg else "")
    return status


def make_events(data, packed=False, weight=None, lattice_mm=0.05):
    """recon_events over a (7, n) float32 array/tensor (SoA planes) or an
    (n, 8) int16 array/tensor of packed records.  The struct keeps `data`
    and `weight` alive."""
    ev = recon_events()
    if isinstance(data, np.ndarray):
        data = np.ascontiguousarray(data)
    elif hasattr(data, "contiguous"):
        data = data.contiguous()
    if packed:
        n = int(data.shape[0])
        ev.fmt = RECON_EV_PACKED_I16_F16
        ev.planes[0] = ptr(data) if n else None
        ev.lattice_mm = lattice_mm
    else:
        n = int(data.shape[1])
        ev.fmt = RECON_EV_F32_SOA
        base = ptr(data)
        for k in range(7):
            ev.planes[k] = base + 4 * k * n if n else None
    ev.n = n
    ev.on_device = 1 if _on_device(data) else 0
    ev.weight = ptr(weight)
    ev._keep = (data, weight)
    return ev


def make_grid(nx, ny, nz, vx, vy, vz, ox, oy, oz):
    return recon_grid(nx, ny, nz, vx, vy, vz, ox, oy, oz)


def regions_array(regions):
    arr = (recon_region * len(regions))()
    for k, (lo, hi) in enumerate(regions):
        arr[k].z_lo, arr[k].z_hi = lo, hi
    return arr


# --------------------------------------------------------------- C names

def recon_create(geometry, grid, tof_fwhm_ps):
    h = C.c_void_p()
    st = load().recon_create(C.byref(geometry), C.byref(grid), float(tof_fwhm_ps), C.byref(h))
    check(None, st)
    return h.value


def recon_destroy(ctx):
    load().recon_destroy(ctx)


def recon_last_error(ctx):
    m = load().recon_last_error(ctx)
    return m.decode() if m else ""


def recon_set_stream(ctx, stream):
    return check(ctx, load().recon_set_stream(ctx, stream))


def recon_set_kernel_window(ctx, k_sigma):
    return check(ctx, load().recon_set_kernel_window(ctx, float(k_sigma)))


def recon_set_gather_bf16(ctx, on):
    return check(ctx, load().recon_set_gather_bf16(ctx, int(bool(on))))


def recon_set_brick_layout(ctx, on):
    return check(ctx, load().recon_set_brick_layout(ctx, int(on)))


PROJ_EXACT = 0
PROJ_SAMPLED = 1
MAX_TOF_SAMPLES = 64


def recon_set_projector(ctx, projector, n_samples=0):
    return check(ctx, load().recon_set_projector(ctx, int(projector), int(n_samples)))


def recon_set_event_order(ctx, order, azimuth_bins=1, polar_bins=1):
    return check(ctx, load().recon_set_event_order(ctx, int(order), int(azimuth_bins), int(polar_bins)))


def recon_set_tiled_pass(ctx, on, lanes=1):
    """0: off; 1: on (cells of >= 256 events); m > 1: on with cells of >= m events.
    lanes: threads per event (1 or 8)."""
    return check(ctx, load().recon_set_tiled_pass(ctx, int(on), int(lanes)))


def recon_set_start_image(ctx, mode):
    """0: uniform start image; 1: starting backprojection."""
    return check(ctx, load().recon_set_start_image(ctx, int(mode)))


def recon_set_subsets(ctx, n_subsets):
    return check(ctx, load().recon_set_subsets(ctx, int(n_subsets)))


def recon_set_median_filter(ctx, on):
    return check(ctx, load().recon_set_median_filter(ctx, int(bool(on))))


def recon_median_filter(ctx, image_in, image_out):
    return check(ctx, load().recon_median_filter(ctx, ptr(image_in), ptr(image_out)))


def recon_preprocess(ctx, events, mu_map, z_reject=1.96, apply=0, weight_out=None, keep_out=None):
    """Attenuation weights and TOF scatter rejection; returns the number of kept events."""
    kept = C.c_int64(0)
    check(ctx, load().recon_preprocess(ctx, C.byref(events) if events is not None else None, ptr(mu_map),
                                       float(z_reject), int(apply), ptr(weight_out), ptr(keep_out), C.byref(kept)))
    return kept.value


def recon_get_tof_samples(ctx):
    """(offsets_mm, weights) float32 arrays of the sampled projector (empty when exact)."""
    t = np.zeros(MAX_TOF_SAMPLES, np.float32)
    w = np.zeros(MAX_TOF_SAMPLES, np.float32)
    n = C.c_int32(0)
    check(ctx, load().recon_get_tof_samples(ctx, MAX_TOF_SAMPLES, t.ctypes.data, w.ctypes.data, C.byref(n)))
    return t[:n.value].copy(), w[:n.value].copy()


def recon_set_launch(ctx, threads_per_block=None, blocks_per_sm=0, chunk_events=0, cached_pieces=0, tail_eval=0,
                     reduction=0):
    if threads_per_block is None:
        return check(ctx, load().recon_set_launch(ctx, None))
    cfg = recon_launch(threads_per_block, blocks_per_sm, chunk_events, cached_pieces, tail_eval, reduction, 0, 1)
    return check(ctx, load().recon_set_launch(ctx, C.byref(cfg)))


def recon_get_launch(ctx):
    """(threads, blocks_per_sm, chunk, cached_pieces, tail_eval, reduction) of the last
    event pass; recon_get_layout gives its image tiling and threads per event."""
    cfg = recon_launch()
    check(ctx, load().recon_get_launch(ctx, C.byref(cfg)))
    return (cfg.threads_per_block, cfg.blocks_per_sm, cfg.chunk_events, cfg.cached_pieces, cfg.tail_eval,
            cfg.reduction)


def recon_get_layout(ctx):
    """(image_tiling, lanes_per_event) of the last MLEM event pass."""
    cfg = recon_launch()
    check(ctx, load().recon_get_launch(ctx, C.byref(cfg)))
    return (cfg.image_tiling, cfg.lanes_per_event)


def recon_set_timing(ctx, on):
    return check(ctx, load().recon_set_timing(ctx, int(bool(on))))


def recon_set_graphs(ctx, on):
    return check(ctx, load().recon_set_graphs(ctx, int(bool(on))))


def recon_set_autotune(ctx, on):
    return check(ctx, load().recon_set_autotune(ctx, int(bool(on))))


def recon_get_info(ctx):
    info = recon_info()
    check(ctx, load().recon_get_info(ctx, C.byref(info)))
    out = {}
    for f, _ in recon_info._fields_:
        v = getattr(info, f)
        out[f] = list(v) if isinstance(v, C.Array) else v
    return out


def recon_get_stats(ctx):
    s = recon_stats()
    check(ctx, load().recon_get_stats(ctx, C.byref(s)))
    return {f: getattr(s, f) for f, _ in recon_stats._fields_}


def recon_reset_stats(ctx):
    return check(ctx, load().recon_reset_stats(ctx))


def recon_sensitivity(ctx, lor, sens_out=None):
    n = int(lor.shape[1]) if lor is not None else 0
    return check(ctx, load().recon_sensitivity(ctx, ptr(lor), n, 1 if _on_device(lor) else 0, ptr(sens_out)))


def recon_set_sensitivity(ctx, sens):
    return check(ctx, load().recon_set_sensitivity(ctx, ptr(sens), 1 if _on_device(sens) else 0))


def recon_load_events(ctx, events):
    return check(ctx, load().recon_load_events(ctx, C.byref(events)))


def recon_forward(ctx, events, image, p_out):
    return check(ctx, load().recon_forward(ctx, C.byref(events) if events is not None else None, ptr(image),
                                           ptr(p_out)))


def recon_backproject(ctx, events, r, image_out):
    return check(ctx, load().recon_backproject(ctx, C.byref(events) if events is not None else None, ptr(r),
                                               ptr(image_out)))


def _check_size(name, arr, need):
    """Host or device buffers the library writes must hold `need` elements."""
    if arr is None:
        return
    size = arr.size if isinstance(arr, np.ndarray) else (arr.numel() if hasattr(arr, "numel") else None)
    if size is not None and size < need:
        raise ValueError(f"{name} holds {size} elements, {need} needed")


def recon_mlem(ctx, events, n_iter, init=None, image_out=None, conservation_out=None):
    if conservation_out is not None:
        _check_size("conservation_out", conservation_out, 2 * int(n_iter) * recon_get_info(ctx)["subsets"])
    return check(ctx, load().recon_mlem(ctx, C.byref(events) if events is not None else None, int(n_iter),
                                        ptr(init), ptr(image_out), ptr(conservation_out)))


def recon_event_pass(ctx, events, image, from_start, C_out):
    """One MLEM event pass into C_out; returns N_eff."""
    _check_size("C_out", C_out, recon_get_info(ctx)["n_vox"])
    n_eff = C.c_double(0.0)
    check(ctx, load().recon_event_pass(ctx, C.byref(events) if events is not None else None, ptr(image),
                                       int(from_start), ptr(C_out), C.byref(n_eff)))
    return n_eff.value


def recon_update(ctx, C_in, image_out=None):
    """The MLEM update from C_in; returns sum_j s_j lambda_j."""
    ssum = C.c_double(0.0)
    check(ctx, load().recon_update(ctx, ptr(C_in), ptr(image_out), C.byref(ssum)))
    return ssum.value


def recon_split_regions(ctx, events, regions, margin_mm, shell_mm, code_out=None, offsets_out=None, idx_out=None):
    arr = regions_array(regions)
    return check(ctx, load().recon_split_regions(ctx, C.byref(events) if events is not None else None, len(regions),
                                                 arr, float(margin_mm), float(shell_mm), ptr(code_out),
                                                 ptr(offsets_out), ptr(idx_out)))


def recon_mlem_regions(ctx, events, regions, margin_mm, shell_mm, n_iter, image_out=None, region_images_out=None,
                       conservation_out=None):
    arr = regions_array(regions)
    return check(ctx, load().recon_mlem_regions(ctx, C.byref(events) if events is not None else None, len(regions),
                                                arr, float(margin_mm), float(shell_mm), int(n_iter), ptr(image_out),
                                                ptr(region_images_out), ptr(conservation_out)))


def recon_set_region_block(ctx, first, count):
    return check(ctx, load().recon_set_region_block(ctx, int(first), int(count)))


def recon_region_slab_voxels(ctx, regions, margin_mm):
    arr = regions_array(regions)
    out = C.c_int64()
    check(ctx, load().recon_region_slab_voxels(ctx, len(regions), arr, float(margin_mm), C.byref(out)))
    return out.value


def recon_debug_fail_alloc(n):
    """Make the n-th device allocation of the library from now on fail (0: disarm)."""
    return check(None, load().recon_debug_fail_alloc(int(n)))


def recon_debug_bounds_violations():
    """Out-of-range voxel indices caught since the last call (-1: normal build)."""
    c = C.c_int64(0)
    check(None, load().recon_debug_bounds_violations(C.byref(c)))
    return c.value


def recon_split_regions_noalloc(grid, events, regions, shell_mm, code_out, offsets_out, idx_out, idx_capacity,
                                stream=None):
    """Allocation-free region split (no context): device events/codes/indices, host offsets."""
    arr = regions_array(regions)
    return check(None, load().recon_split_regions_noalloc(C.byref(grid), C.byref(events), len(regions), arr,
                                                          float(shell_mm), ptr(code_out), ptr(offsets_out),
                                                          ptr(idx_out), int(idx_capacity), stream))


# ------------------------------------------------------------ convenience

class Context:
    """Owns one recon_ctx; methods forward to the functions above."""

    def __init__(self, geometry, grid, tof_fwhm_ps=300.0):
        if not isinstance(geometry, recon_geometry):
            geometry = recon_geometry(*geometry)
        if not isinstance(grid, recon_grid):
            grid = recon_grid(*grid)
        self.grid = grid
        self.handle = recon_create(geometry, grid, tof_fwhm_ps)

    @property
    def n_vox(self):
        return self.grid.nx * self.grid.ny * self.grid.nz

    def close(self):
        if self.handle:
            recon_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __getattr__(self, name):
        fn = globals().get("recon_" + name)
        if fn is None:
            raise AttributeError(name)
        return lambda *a, **k: fn(self.handle, *a, **k)
