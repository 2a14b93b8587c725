"""Python binding of libbh (ctypes), one function per C-ABI entry point.

Argument marshalling only: every step of the render and of the precompute
runs in the CUDA kernels of ``libbh.so``.  Device buffers are passed as raw
device pointers (``int``) or as torch CUDA tensors; streams as
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or ``None``.
There is no CPU fallback: if ``libbh.so`` is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
LIBPATH = HERE / "libbh.so"

BH_OK, BH_ERR_INVALID_ARG, BH_ERR_CUDA, BH_ERR_OOM, BH_ERR_BUSY, BH_ERR_NOT_READY, \
    BH_ERR_TIMEOUT, BH_ERR_DEVICE_STATUS = range(8)
BH_F32, BH_F16, BH_BF16 = 0, 1, 2
STATUS_NAMES = {0: "BH_OK", 1: "BH_ERR_INVALID_ARG", 2: "BH_ERR_CUDA", 3: "BH_ERR_OOM",
                4: "BH_ERR_BUSY", 5: "BH_ERR_NOT_READY", 6: "BH_ERR_TIMEOUT",
                7: "BH_ERR_DEVICE_STATUS"}
NDBG = 20


class BhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("r", C.c_double), ("theta", C.c_double), ("phi", C.c_double),
                ("v", C.c_double * 3), ("orient", C.c_double * 9), ("fov_y", C.c_double),
                ("width", C.c_int), ("height", C.c_int)]


class Disc(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_out", C.c_double), ("t_peak_K", C.c_double),
                ("density", C.c_double), ("enabled", C.c_int), ("particles", C.c_void_p),
                ("time", C.c_double)]


class Shading(C.Structure):
    _fields_ = [("exposure_disc", C.c_float), ("exposure_stars", C.c_float)]


class TableDesc(C.Structure):
    _fields_ = [("d_n", C.c_int), ("u_ne", C.c_int), ("u_nphi", C.c_int), ("storage", C.c_int)]


class Orbit(C.Structure):
    _fields_ = [("t", C.c_double), ("r", C.c_double), ("psi", C.c_double), ("rdot", C.c_double),
                ("e", C.c_double), ("l", C.c_double), ("chi", C.c_double),
                ("orient", C.c_double * 9), ("fov_y", C.c_double), ("width", C.c_int),
                ("height", C.c_int)]


class Star(C.Structure):
    _fields_ = [("dir", C.c_float * 3), ("lum", C.c_float), ("temp_K", C.c_float)]


_lib = None
_vp = C.c_void_p


def lib():
    """Load libbh.so (built by ``__graft_entry__.build()`` or ``build.py``)."""
    global _lib
    if _lib is None:
        if not LIBPATH.exists():
            raise BhError(BH_ERR_CUDA, f"{LIBPATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(str(LIBPATH))
        P = C.POINTER
        sig = {
            "bh_create": [C.c_int, C.c_size_t, P(_vp)],
            "bh_destroy": None,
            "bh_precompute_tables": [_vp, P(TableDesc), _vp, P(_vp)],
            "bh_tables_upload": [_vp, P(TableDesc), P(C.c_double), P(C.c_double), _vp, P(_vp)],
            "bh_tables_copy_out": [_vp, P(C.c_double), P(C.c_double)],
            "bh_tables_upload_time": [_vp, P(C.c_double), P(C.c_double), _vp],
            "bh_disc_particles_create": [_vp, P(C.c_double), C.c_int, P(_vp)],
            "bh_tables_save": [_vp, C.c_char_p],
            "bh_tables_load": [_vp, C.c_char_p, _vp, P(_vp)],
            "bh_cubemap_save": [_vp, C.c_char_p],
            "bh_cubemap_load": [_vp, C.c_char_p, _vp, P(_vp)],
            "bh_tables_copy_time": [_vp, P(C.c_double), P(C.c_double)],
            "bh_tables_copy_colour": [_vp, P(C.c_float), P(C.c_float)],
            "bh_build_star_cubemap": [_vp, _vp, C.c_longlong, C.c_int, C.c_int, C.c_int, _vp,
                                      P(_vp)],
            "bh_cubemap_copy_out": [_vp, P(C.c_uint16), C.c_longlong],
            "bh_build_star_cubemap_noalloc": [_vp, C.c_longlong, C.c_int, C.c_int, _vp, _vp],
            "bh_render": [_vp, _vp, _vp, P(Camera), P(Disc), P(Shading), _vp, _vp],
            "bh_render_debug": [_vp, _vp, _vp, P(Camera), P(Disc), P(Shading), _vp, _vp, _vp],
            "bh_render_to_host": [_vp, _vp, _vp, P(Camera), P(Disc), P(Shading), _vp, _vp],
            "bh_render_to_host_rgb": [_vp, _vp, _vp, P(Camera), P(Disc), P(Shading), _vp, _vp],
            "bh_render_to_host_async": [_vp, _vp, _vp, P(Camera), P(Disc), P(Shading), _vp, C.c_int, _vp,
                                        P(C.c_ulonglong)],
            "bh_host_wait": [_vp, C.c_ulonglong],
            "bh_render_batch": [_vp, _vp, _vp, C.c_int, P(Camera), P(Disc), P(Shading),
                                P(_vp), _vp],
            "bh_autotune_batch": [_vp, _vp, _vp, C.c_int, P(Camera), P(Disc), P(Shading),
                                  P(_vp), P(C.c_int)],
            "bh_orbit_init": [C.c_double, C.c_double, C.c_double, C.c_double, P(C.c_double),
                              C.c_double, C.c_int, C.c_int, P(Orbit)],
            "bh_orbit_camera": [P(Orbit), P(Camera)],
            "bh_orbits_advance": [_vp, _vp, C.c_int, C.c_double, C.c_int, _vp],
            "bh_render_orbits": [_vp, _vp, _vp, C.c_int, _vp, P(Disc), P(Shading), P(_vp), _vp],
            "bh_serve_submit": [_vp, _vp, _vp, C.c_int, P(Camera), P(Disc), P(Shading), _vp,
                                P(C.c_ulonglong)],
            "bh_serve_poll": [_vp, C.c_ulonglong, C.c_int, P(C.c_double)],
            "bh_serve_submit_orbit": [_vp, _vp, _vp, C.c_int, _vp, C.c_double, C.c_int, C.c_int, C.c_int,
                                      P(Disc), P(Shading), _vp, P(C.c_ulonglong)],
            "bh_serve_flush": [_vp],
            "bh_check_status": [_vp, _vp],
            "bh_measure_issue_rates": [C.c_int, P(C.c_double)],
            "bh_measure_host_link": [C.c_int, C.c_size_t, P(C.c_double)],
            "bh_bloom_weights": [C.c_double, C.c_int, C.c_int, P(C.c_double)],
            "bh_bloom": [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, P(C.c_double), _vp],
            "bh_inject_fault": [_vp, C.c_int],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            if args is None:
                fn.argtypes = [_vp]
                fn.restype = None
            else:
                fn.argtypes = args
                fn.restype = C.c_int
        L.bh_last_error.restype = C.c_char_p
        L.bh_last_error.argtypes = []
        L.bh_kernel_launches.restype = C.c_longlong
        L.bh_kernel_launches.argtypes = [_vp]
        L.bh_cubemap_records.restype = C.c_longlong
        L.bh_cubemap_records.argtypes = [C.c_int]
        L.bh_tables_free.argtypes = [_vp]
        L.bh_tables_free.restype = None
        L.bh_cubemap_free.argtypes = [_vp]
        L.bh_cubemap_free.restype = None
        L.bh_disc_particles_free.argtypes = [_vp]
        L.bh_disc_particles_free.restype = None
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return [n for n in dir(lib()) if n.startswith("bh_")]


def _check(status: int, allow=()):
    if status != BH_OK and status not in allow:
        raise BhError(status, lib().bh_last_error().decode())
    return status


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor, or an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError(f"not a stream: {type(s)}")


# ---------------------------------------------------------------------------
# struct helpers
# ---------------------------------------------------------------------------

def make_camera(cam: dict) -> Camera:
    c = Camera()
    c.r, c.theta, c.phi = cam["r"], cam["theta"], cam["phi"]
    for k in range(3):
        c.v[k] = cam["v"][k]
    o = np.asarray(cam["orient"], dtype=np.float64).reshape(9)
    for k in range(9):
        c.orient[k] = o[k]
    c.fov_y, c.width, c.height = cam["fov_y"], cam["width"], cam["height"]
    return c


def make_disc(d: dict) -> Disc:
    """d may carry "particles_handle" (from bh_disc_particles_create) and "time"."""
    x = Disc()
    x.r_in, x.r_out, x.t_peak_K, x.density = d["r_in"], d["r_out"], d["t_peak"], d["density"]
    x.enabled = int(d.get("enabled", 1))
    x.particles = d.get("particles_handle")
    x.time = float(d.get("time", 0.0))
    return x


def make_shading(exposure_disc=1.0, exposure_stars=0.01) -> Shading:
    return Shading(exposure_disc, exposure_stars)


def _as(obj, maker):
    return obj if not isinstance(obj, dict) else maker(obj)


# ---------------------------------------------------------------------------
# C-ABI entry points
# ---------------------------------------------------------------------------

def bh_last_error() -> str:
    return lib().bh_last_error().decode()


def bh_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    out = _vp()
    _check(lib().bh_create(device, hbm_budget_bytes, C.byref(out)))
    return out.value


def bh_destroy(ctx: int) -> None:
    lib().bh_destroy(ctx)


BH_FAULT_TABLE_WAIT = 1
BH_FAULT_BLOOM_BARRIER = 2


def bh_check_status(ctx: int, stream=None) -> int:
    """BH_OK, or raises BhError (BH_ERR_TIMEOUT / BH_ERR_DEVICE_STATUS)."""
    return _check(lib().bh_check_status(ctx, _stream(stream)))


def bh_bloom_weights(fov_y: float, height: int, levels: int) -> np.ndarray:
    """Per-level weights of the bloom (share of the PSF's energy per octave of radius)."""
    w = np.zeros(levels + 1)
    _check(lib().bh_bloom_weights(fov_y, height, levels, w.ctypes.data_as(C.POINTER(C.c_double))))
    return w


def bh_bloom(ctx, inp, out, width: int, height: int, weights, stream=None) -> None:
    """Bloom of a (height, width, 4) float32 CUDA frame into `out` (may be `inp`)."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    _check(lib().bh_bloom(ctx, _ptr(inp), _ptr(out), width, height, w.size - 1,
                          w.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))


def bh_measure_issue_rates(device: int = 0) -> dict:
    """SM issue rates measured by the library's microbenchmark kernels."""
    o = (C.c_double * 5)()
    _check(lib().bh_measure_issue_rates(device, o))
    return {"fp32_fma_per_sm_clk": o[0], "ffma2_fma_per_sm_clk": o[1], "mufu_per_sm_clk": o[2],
            "sms": int(o[3]), "sm_mhz": o[4]}


def bh_measure_host_link(device: int = 0, nbytes: int = 1 << 25) -> dict:
    """Device-to-pinned-host bandwidth (GB/s) by the copy engine and by kernel stores."""
    o = (C.c_double * 2)()
    _check(lib().bh_measure_host_link(device, nbytes, o))
    return {"copy_engine_gbs": o[0], "kernel_stores_gbs": o[1], "bytes": nbytes}


def bh_inject_fault(ctx: int, kind: int = BH_FAULT_TABLE_WAIT) -> None:
    _check(lib().bh_inject_fault(ctx, kind))


def bh_kernel_launches(ctx: int) -> int:
    return lib().bh_kernel_launches(ctx)


def bh_precompute_tables(ctx: int, d_n=512, u_ne=64, u_nphi=32, storage=BH_F32,
                         stream=None) -> int:
    desc = TableDesc(d_n, u_ne, u_nphi, storage)
    out = _vp()
    _check(lib().bh_precompute_tables(ctx, C.byref(desc), _stream(stream), C.byref(out)))
    return out.value


def bh_tables_upload(ctx: int, D: np.ndarray, U: np.ndarray, storage=BH_F32, stream=None) -> int:
    D = np.ascontiguousarray(D, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    desc = TableDesc(D.shape[0], U.shape[1], U.shape[0], storage)
    out = _vp()
    _check(lib().bh_tables_upload(ctx, C.byref(desc), D.ctypes.data_as(C.POINTER(C.c_double)),
                                  U.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream),
                                  C.byref(out)))
    return out.value


def bh_tables_copy_out(tables: int, d_n: int, u_ne: int, u_nphi: int):
    D = np.zeros((d_n, d_n))
    U = np.zeros((u_nphi, u_ne))
    _check(lib().bh_tables_copy_out(tables, D.ctypes.data_as(C.POINTER(C.c_double)),
                                    U.ctypes.data_as(C.POINTER(C.c_double))))
    return D, U


def bh_tables_upload_time(tables: int, DT: np.ndarray, UT: np.ndarray, stream=None) -> None:
    DT = np.ascontiguousarray(DT, dtype=np.float64)
    UT = np.ascontiguousarray(UT, dtype=np.float64)
    _check(lib().bh_tables_upload_time(tables, DT.ctypes.data_as(C.POINTER(C.c_double)),
                                       UT.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))


def bh_tables_copy_time(tables: int, d_n: int, u_ne: int, u_nphi: int):
    """Regularised-time channels (DT, UT), same layouts as D and U."""
    DT = np.zeros((d_n, d_n))
    UT = np.zeros((u_nphi, u_ne))
    _check(lib().bh_tables_copy_time(tables, DT.ctypes.data_as(C.POINTER(C.c_double)),
                                     UT.ctypes.data_as(C.POINTER(C.c_double))))
    return DT, UT


def bh_disc_particles_create(ctx: int, particles) -> int:
    """particles: (n, 3) rows (u1, u2, phi0) of the animated disc."""
    arr = np.ascontiguousarray(particles, dtype=np.float64).reshape(-1, 3)
    out = _vp()
    _check(lib().bh_disc_particles_create(ctx, arr.ctypes.data_as(C.POINTER(C.c_double)), arr.shape[0],
                                          C.byref(out)))
    return out.value


def bh_disc_particles_free(p: int) -> None:
    lib().bh_disc_particles_free(p)


def bh_tables_save(tables: int, path) -> None:
    _check(lib().bh_tables_save(tables, str(path).encode()))


def bh_tables_load(ctx: int, path, stream=None) -> int:
    out = _vp()
    _check(lib().bh_tables_load(ctx, str(path).encode(), _stream(stream), C.byref(out)))
    return out.value


def bh_cubemap_save(cube: int, path) -> None:
    _check(lib().bh_cubemap_save(cube, str(path).encode()))


def bh_cubemap_load(ctx: int, path, stream=None) -> int:
    out = _vp()
    _check(lib().bh_cubemap_load(ctx, str(path).encode(), _stream(stream), C.byref(out)))
    return out.value


def bh_tables_copy_colour(tables: int):
    Ct = np.zeros((64, 32, 64, 4), dtype=np.float32)
    dt = np.zeros((1024, 4), dtype=np.float32)
    _check(lib().bh_tables_copy_colour(tables, Ct.ctypes.data_as(C.POINTER(C.c_float)),
                                       dt.ctypes.data_as(C.POINTER(C.c_float))))
    return Ct, dt


def bh_tables_free(tables: int) -> None:
    lib().bh_tables_free(tables)


def bh_build_star_cubemap(ctx: int, stars, face_size: int, storage=BH_F16, stream=None) -> int:
    """stars: (n, 5) float32 numpy array (host) or a torch CUDA tensor (device)."""
    out = _vp()
    if hasattr(stars, "is_cuda") and stars.is_cuda:
        assert stars.dtype.itemsize == 4 and stars.shape[-1] == 5 and stars.is_contiguous()
        n, ptr, on_dev = stars.shape[0], stars.data_ptr(), 1
        keep = stars
    else:
        keep = np.ascontiguousarray(stars, dtype=np.float32)
        assert keep.ndim == 2 and keep.shape[1] == 5
        n, ptr, on_dev = keep.shape[0], keep.ctypes.data, 0
    _check(lib().bh_build_star_cubemap(ctx, ptr, n, face_size, storage, on_dev, _stream(stream),
                                       C.byref(out)))
    del keep
    return out.value


def bh_build_star_cubemap_noalloc(stars, face_size: int, storage, records, stream=None) -> None:
    """Allocation-free cube-map build: stars is a (n, 5) float32 CUDA tensor,
    records a caller-owned CUDA tensor of bh_cubemap_records(face_size) x 4
    uint16 (or int16); face_size <= 128.  Runs on the current device."""
    import torch
    assert stars.is_cuda and stars.is_contiguous() and stars.shape[-1] == 5
    assert stars.dtype == torch.float32, "stars must be float32 (bh_star: dir[3], lum, temp_K)"
    assert records.is_cuda and records.is_contiguous() and records.element_size() == 2
    assert records.numel() >= 4 * bh_cubemap_records(face_size)
    cur = torch.cuda.current_device()
    assert stars.device.index == cur and records.device.index == cur, \
        "stars and records must be on the current CUDA device"
    _check(lib().bh_build_star_cubemap_noalloc(stars.data_ptr() if stars.shape[0] else None,
                                               stars.shape[0], face_size, storage,
                                               records.data_ptr(), _stream(stream)))


def bh_cubemap_records(face_size: int) -> int:
    return lib().bh_cubemap_records(face_size)


def bh_cubemap_copy_out(cube: int, face_size: int) -> np.ndarray:
    n = bh_cubemap_records(face_size)
    rec = np.zeros((n, 4), dtype=np.uint16)
    _check(lib().bh_cubemap_copy_out(cube, rec.ctypes.data_as(C.POINTER(C.c_uint16)), n))
    return rec


def bh_cubemap_free(cube: int) -> None:
    lib().bh_cubemap_free(cube)


def bh_render(ctx, tables, cube, camera, disc, shading, out, stream=None) -> None:
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    _check(lib().bh_render(ctx, tables, cube, C.byref(cam), C.byref(d), C.byref(shading),
                           _ptr(out), _stream(stream)))


def bh_render_debug(ctx, tables, cube, camera, disc, shading, out, dbg, stream=None) -> None:
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    _check(lib().bh_render_debug(ctx, tables, cube, C.byref(cam), C.byref(d), C.byref(shading),
                                 _ptr(out), _ptr(dbg), _stream(stream)))


def bh_render_to_host(ctx, tables, cube, camera, disc, shading, out_host: np.ndarray,
                      stream=None) -> None:
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    if isinstance(out_host, np.ndarray):
        assert out_host.dtype == np.float32 and out_host.flags["C_CONTIGUOUS"]
        assert out_host.size >= cam.width * cam.height * 4
        p = out_host.ctypes.data
    else:  # pinned torch CPU tensor
        assert out_host.numel() >= cam.width * cam.height * 4
        p = out_host.data_ptr()
    _check(lib().bh_render_to_host(ctx, tables, cube, C.byref(cam), C.byref(d),
                                   C.byref(shading), p, _stream(stream)))


def bh_render_to_host_rgb(ctx, tables, cube, camera, disc, shading, out_host, stream=None) -> None:
    """As bh_render_to_host, into packed linear RGB (height, width, 3) float32."""
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    if isinstance(out_host, np.ndarray):
        assert out_host.dtype == np.float32 and out_host.flags["C_CONTIGUOUS"]
        assert out_host.size >= cam.width * cam.height * 3
        p = out_host.ctypes.data
    else:  # torch CPU tensor (pinned for the direct path)
        assert out_host.dtype.itemsize == 4 and out_host.is_contiguous()
        assert out_host.numel() >= cam.width * cam.height * 3
        p = out_host.data_ptr()
    _check(lib().bh_render_to_host_rgb(ctx, tables, cube, C.byref(cam), C.byref(d),
                                       C.byref(shading), p, _stream(stream)))


def bh_render_to_host_async(ctx, tables, cube, camera, disc, shading, out_host, rgb=True, stream=None) -> int:
    """Enqueue a frame to pinned host memory (packed RGB (height, width, 3) or
    RGBA (height, width, 4) float32) with two frames in flight; returns the
    frame's ticket for bh_host_wait.  out_host must stay untouched until then."""
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    ch = 3 if rgb else 4
    assert out_host.dtype.itemsize == 4 and out_host.is_contiguous()
    assert out_host.numel() >= cam.width * cam.height * ch
    t = C.c_ulonglong(0)
    _check(lib().bh_render_to_host_async(ctx, tables, cube, C.byref(cam), C.byref(d), C.byref(shading),
                                         out_host.data_ptr(), 1 if rgb else 0, _stream(stream), C.byref(t)))
    return t.value


def bh_host_wait(ctx, ticket: int) -> None:
    """Block until frame `ticket` of bh_render_to_host_async is in host memory."""
    _check(lib().bh_host_wait(ctx, C.c_ulonglong(ticket)))


def _cams(cameras):
    arr = (Camera * len(cameras))()
    for k, c in enumerate(cameras):
        arr[k] = _as(c, make_camera)
    return arr


def bh_render_batch(ctx, tables, cube, cameras, disc, shading, outs, stream=None) -> None:
    n = len(cameras)
    cams = _cams(cameras)
    ptrs = (_vp * n)(*[_ptr(o) for o in outs])
    d = _as(disc, make_disc)
    _check(lib().bh_render_batch(ctx, tables, cube, n, cams, C.byref(d), C.byref(shading), ptrs,
                                 _stream(stream)))


def bh_autotune_batch(ctx, tables, cube, cameras, disc, shading, outs) -> int:
    n = len(cameras)
    cams = _cams(cameras)
    ptrs = (_vp * n)(*[_ptr(o) for o in outs])
    d = _as(disc, make_disc)
    chosen = C.c_int(-1)
    _check(lib().bh_autotune_batch(ctx, tables, cube, n, cams, C.byref(d), C.byref(shading),
                                   ptrs, C.byref(chosen)))
    return chosen.value


def bh_orbit_init(r0, delta0, v0, chi, orient=None, fov_y=1.0471975511965976, width=256,
                  height=256) -> Orbit:
    o = Orbit()
    op = None
    if orient is not None:
        arr = (C.c_double * 9)(*np.asarray(orient, dtype=np.float64).reshape(9))
        op = C.cast(arr, C.POINTER(C.c_double))
    _check(lib().bh_orbit_init(r0, delta0, v0, chi, op, fov_y, width, height, C.byref(o)))
    return o


def bh_orbit_camera(orbit: Orbit) -> Camera:
    c = Camera()
    _check(lib().bh_orbit_camera(C.byref(orbit), C.byref(c)))
    return c


def orbits_to_bytes(orbits) -> bytes:
    """Packed bh_orbit array (copy it into a device buffer)."""
    arr = (Orbit * len(orbits))(*orbits)
    return bytes(arr)


def bh_orbits_advance(ctx, orbits_device, n, dtau, steps=8, stream=None) -> None:
    _check(lib().bh_orbits_advance(ctx, _ptr(orbits_device), n, dtau, steps, _stream(stream)))


def bh_render_orbits(ctx, tables, cube, n, orbits_device, disc, shading, outs, stream=None) -> None:
    ptrs = (_vp * n)(*[_ptr(o) for o in outs])
    d = _as(disc, make_disc)
    _check(lib().bh_render_orbits(ctx, tables, cube, n, _ptr(orbits_device), C.byref(d),
                                  C.byref(shading), ptrs, _stream(stream)))


def camera_to_dict(c: Camera) -> dict:
    return {"r": c.r, "theta": c.theta, "phi": c.phi, "v": tuple(c.v[:]),
            "orient": tuple(tuple(c.orient[3 * i:3 * i + 3]) for i in range(3)),
            "fov_y": c.fov_y, "width": c.width, "height": c.height}


def bh_serve_submit(ctx, tables, cube, viewer, camera, disc, shading, out):
    """Returns (status, ticket); status is BH_OK or BH_ERR_BUSY (admission refused)."""
    cam = _as(camera, make_camera)
    d = _as(disc, make_disc)
    t = C.c_ulonglong(0)
    st = _check(lib().bh_serve_submit(ctx, tables, cube, viewer, C.byref(cam), C.byref(d),
                                      C.byref(shading), _ptr(out), C.byref(t)),
                allow=(BH_ERR_BUSY,))
    return st, t.value


def bh_serve_submit_orbit(ctx, tables, cube, viewer, orbit_device_ptr, dtau, steps, width, height, disc,
                          shading, out):
    """orbit_device_ptr: device address of the viewer's bh_orbit.  Returns
    (status, ticket) as bh_serve_submit."""
    d = _as(disc, make_disc)
    t = C.c_ulonglong(0)
    st = _check(lib().bh_serve_submit_orbit(ctx, tables, cube, viewer, orbit_device_ptr, dtau, steps, width,
                                            height, C.byref(d), C.byref(shading), _ptr(out), C.byref(t)),
                allow=(BH_ERR_BUSY,))
    return st, t.value


def bh_serve_poll(ctx, ticket, timeout_us=0):
    """Returns (status, latency_ms); status is BH_OK or BH_ERR_NOT_READY."""
    lat = C.c_double(0.0)
    st = _check(lib().bh_serve_poll(ctx, ticket, timeout_us, C.byref(lat)),
                allow=(BH_ERR_NOT_READY,))
    return st, lat.value


def bh_serve_flush(ctx) -> None:
    _check(lib().bh_serve_flush(ctx))
