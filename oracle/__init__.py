"""CPU FP64 oracle for the table-driven Schwarzschild beam tracer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2010_08735_gb300``) never imports, links
or runs anything here, and this package imports nothing from the product.

The arithmetic lives in ``bh_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes and numpy.  Each wrapped function names the passage of the paper it
follows (E. Bruneton, "Real-time High-Quality Rendering of Non-Rotating Black
Holes", 2020).

Colour: the observer (piecewise-Gaussian colour-matching functions) is pinned
in absolute terms through ``blackbody_xyz``, whose chromaticities lie on the
published Planckian locus within the fit's accuracy; the C(xy, D)
chromaticity-to-spectrum choice (``colour_table``, the paper's A1 = A2 = 0) is
a project definition whose internal consistency (black-body temperature shift)
is pinned -- parity unpinned for that choice itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "bh_oracle.c"
LIB = HERE / "liboracle.so"

MU = 4.0 / 27.0
NDBG = 29

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", str(tmp), str(SRC), "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class Camera(C.Structure):
    _fields_ = [("r", C.c_double), ("theta", C.c_double), ("phi", C.c_double),
                ("v", C.c_double * 3), ("orient", C.c_double * 9),
                ("fov_y", C.c_double), ("width", C.c_int), ("height", C.c_int)]


class Disc(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_out", C.c_double), ("t_peak", C.c_double),
                ("density", C.c_double), ("enabled", C.c_int),
                ("particles", C.POINTER(C.c_double)), ("n_particles", C.c_int),
                ("time", C.c_double)]


class Scene(C.Structure):
    _fields_ = [("D", C.POINTER(C.c_double)), ("d_n", C.c_int),
                ("U", C.POINTER(C.c_double)), ("u_ne", C.c_int), ("u_nphi", C.c_int),
                ("DT", C.POINTER(C.c_double)), ("UT", C.POINTER(C.c_double)),
                ("C", C.POINTER(C.c_double)), ("c_nx", C.c_int), ("c_ny", C.c_int),
                ("c_nd", C.c_int),
                ("disc_ln", C.POINTER(C.c_double)), ("disc_n", C.c_int),
                ("cube", C.POINTER(C.c_uint16)), ("cube_n", C.c_int), ("cube_dtype", C.c_int)]


class Orbit(C.Structure):
    _fields_ = [("t", C.c_double), ("r", C.c_double), ("psi", C.c_double), ("rdot", C.c_double),
                ("e", C.c_double), ("l", C.c_double), ("chi", C.c_double)]


_D = C.POINTER(C.c_double)


LIB_COUNT = HERE / "liboracle_count.so"
_lib_count = None
COUNT_CLASSES = ("add", "mul", "div", "sqrt", "transcendental", "compare", "other",
                 "fetch_D", "fetch_U", "fetch_C", "fetch_disc", "fetch_cube")


def build_count(force: bool = False) -> Path:
    """Compile the counting build (op_count.cpp: this oracle as C++ with
    counting doubles) into ``oracle/liboracle_count.so``."""
    deps = [SRC, HERE / "op_count.cpp", HERE / "op_count.hpp"]
    if force or not LIB_COUNT.exists() or any(LIB_COUNT.stat().st_mtime < d.stat().st_mtime for d in deps):
        tmp = LIB_COUNT.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", str(tmp), str(HERE / "op_count.cpp"), "-lm", "-lpthread"]
        subprocess.run(cmd, check=True, cwd=str(HERE))
        os.replace(tmp, LIB_COUNT)
    return LIB_COUNT


def lib_count():
    global _lib_count
    if _lib_count is None:
        build_count()
        L = C.CDLL(str(LIB_COUNT))
        L.orc_render.restype = C.c_int
        L.orc_render.argtypes = [C.POINTER(Camera), C.POINTER(Disc), C.c_double, C.c_double,
                                 C.POINTER(Scene), C.c_int, C.c_int, C.c_int, C.c_int,
                                 _D, _D, C.POINTER(C.c_longlong)]
        L.orc_count_reset.restype = None
        L.orc_count_reset.argtypes = [C.c_longlong]
        L.orc_count_read.restype = None
        L.orc_count_read.argtypes = [C.POINTER(C.c_longlong)]
        _lib_count = L
    return _lib_count


def count_render(cam: dict, disc: dict, tables: "SceneTables", exposure_disc=1.0, exposure_stars=0.01,
                 y0=0, y1=None, nthreads=None):
    """The oracle's render of rows [y0, y1) in its counting build: returns
    (rgba, counts), counts a dict of the per-pixel work tallied by class
    (COUNT_CLASSES), the unique cube-map records read ("unique_cube_records")
    and the unique occupied ones ("unique_cube_records_occupied")."""
    L = lib_count()
    c = make_camera(cam)
    d = make_disc(disc)
    y1 = cam["height"] if y1 is None else y1
    out = np.zeros((y1 - y0, cam["width"], 4))
    tex = C.c_longlong(0)
    s = tables.scene()
    nrec = cube_records(tables.cube_n) if tables.cube is not None else 0
    L.orc_count_reset(nrec)
    rc = L.orc_render(C.byref(c), C.byref(d), exposure_disc, exposure_stars, C.byref(s), y0, y1, -1,
                      nthreads or (os.cpu_count() or 1), _dp(out), None, C.byref(tex))
    if rc:
        raise ValueError(f"orc_render (counting) failed ({rc})")
    raw = (C.c_longlong * (len(COUNT_CLASSES) + 2))()
    L.orc_count_read(raw)
    counts = dict(zip(COUNT_CLASSES, raw[:len(COUNT_CLASSES)]))
    counts["unique_cube_records"] = raw[len(COUNT_CLASSES)]
    counts["unique_cube_records_occupied"] = raw[len(COUNT_CLASSES) + 1]
    counts["pixels"] = (y1 - y0) * cam["width"]
    return out, counts


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        sig = {
            "orc_apsis": (C.c_double, [C.c_double]),
            "orc_d_e2_of_x": (C.c_double, [C.c_double]),
            "orc_d_u_of_y": (C.c_double, [C.c_double, C.c_double]),
            "orc_u_e2_of_x": (C.c_double, [C.c_double]),
            "orc_u_phi_of_y": (C.c_double, [C.c_double, C.c_double]),
            "orc_tables_exact": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, _D, _D]),
            "orc_tables_exact2": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, _D, _D, _D, _D]),
            "orc_time_of_R": (C.c_double, [C.c_double, C.c_double]),
            "orc_time_at_phi": (None, [C.c_double, C.c_double, C.c_double, _D]),
            "orc_trace_ray2": (None, [_D, _D, C.c_int, _D, _D, C.c_int, C.c_int, C.c_double,
                                      C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, _D]),
            "orc_u_of_phi": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_state_at_phi": (None, [C.c_double, C.c_double, C.c_double, _D]),
            "orc_apsis_deflection": (C.c_double, [C.c_double, C.c_double]),
            "orc_d_lookup": (C.c_double, [_D, C.c_int, C.c_double, C.c_double]),
            "orc_u_lookup": (C.c_double, [_D, C.c_int, C.c_int, C.c_double, C.c_double]),
            "orc_trace_ray": (None, [_D, C.c_int, _D, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_double, C.c_int, C.c_double, C.c_double, _D]),
            "orc_cmf": (None, [C.c_double, _D]),
            "orc_planck": (C.c_double, [C.c_double, C.c_double]),
            "orc_blackbody_xyz": (None, [C.c_double, _D]),
            "orc_xyz_to_rgb_matrix": (None, [_D]),
            "orc_disc_colour_table": (C.c_int, [C.c_int, _D]),
            "orc_disc_xyz": (None, [_D, C.c_int, C.c_double, _D]),
            "orc_colour_table": (C.c_int, [C.c_int, C.c_int, C.c_int, _D]),
            "orc_decode16": (C.c_double, [C.c_uint16, C.c_int]),
            "orc_encode16": (C.c_uint16, [C.c_double, C.c_int]),
            "orc_cube_level_offset": (C.c_longlong, [C.c_int, C.c_int]),
            "orc_cube_levels": (C.c_int, [C.c_int]),
            "orc_star_xyz": (None, [C.c_double, C.c_double, C.POINTER(C.c_float)]),
            "orc_build_cubemap": (C.c_int, [C.POINTER(C.c_float), C.c_longlong, C.c_int, C.c_int,
                                            C.POINTER(C.c_uint16)]),
            "orc_beam": (None, [C.POINTER(Camera), C.c_double, C.c_double, _D]),
            "orc_disc_doppler": (C.c_double, [C.c_double] * 5),
            "orc_disc_temperature": (C.c_double, [C.c_double, C.c_double]),
            "orc_render": (C.c_int, [C.POINTER(Camera), C.POINTER(Disc), C.c_double, C.c_double,
                                     C.POINTER(Scene), C.c_int, C.c_int, C.c_int, C.c_int,
                                     _D, _D, C.POINTER(C.c_longlong)]),
            "orc_bruteforce_ray": (C.c_int, [_D, _D, C.c_double, C.c_double, C.c_double, _D]),
            "orc_ellipk": (C.c_double, [C.c_double]),
            "orc_particle_point": (None, [_D, C.c_double, C.c_double, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
            "orc_disc_density": (C.c_double, [_D, C.c_int, C.c_double, C.c_double, C.c_double,
                                              C.c_double]),
            "orc_orbit_init": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.POINTER(Orbit)]),
            "orc_orbit_advance": (None, [C.POINTER(Orbit), C.c_double, C.c_int]),
            "orc_orbit_camera": (None, [C.POINTER(Orbit), _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


# --------------------------------------------------------------------------
# Tables (Algorithm 1 PRECOMPUTE, Appendix A mappings)
# --------------------------------------------------------------------------

def apsis(e2: float) -> float:
    """Eq. uapsis."""
    return lib().orc_apsis(e2)


def d_e2_of_x(x: float) -> float:
    return lib().orc_d_e2_of_x(x)


def d_u_of_y(e2: float, y: float) -> float:
    return lib().orc_d_u_of_y(e2, y)


def u_e2_of_x(x: float) -> float:
    return lib().orc_u_e2_of_x(x)


def u_phi_of_y(e2: float, y: float) -> float:
    return lib().orc_u_phi_of_y(e2, y)


def tables_exact(d_n: int = 512, u_ne: int = 64, u_nphi: int = 32, h0: float = 1e-3):
    """D (d_n x d_n, [u-index, e-index]) and U (u_nphi x u_ne, [phi-index,
    e-index]) sampled at texel centres: Algorithm 1 with RK4 in phi."""
    D = np.zeros((d_n, d_n))
    U = np.zeros((u_nphi, u_ne))
    rc = lib().orc_tables_exact(d_n, u_ne, u_nphi, h0, _dp(D), _dp(U))
    if rc:
        raise ValueError(f"orc_tables_exact failed ({rc})")
    return D, U


def tables_exact_t(d_n: int = 512, u_ne: int = 64, u_nphi: int = 32, h0: float = 1e-3):
    """As tables_exact, plus the regularised time channels R = t + 1/u -
    ln(u/(1-u)) of D and U (same layouts): returns D, U, DT, UT."""
    D = np.zeros((d_n, d_n)); U = np.zeros((u_nphi, u_ne))
    DT = np.zeros((d_n, d_n)); UT = np.zeros((u_nphi, u_ne))
    rc = lib().orc_tables_exact2(d_n, u_ne, u_nphi, h0, _dp(D), _dp(U), _dp(DT), _dp(UT))
    if rc:
        raise ValueError(f"orc_tables_exact2 failed ({rc})")
    return D, U, DT, UT


def time_of_R(R: float, u: float) -> float:
    return lib().orc_time_of_R(R, u)


def time_at_phi(e2: float, phi: float, h0: float = 1e-4):
    """(u, du/dphi, R, t) at angle phi on the ray from infinity."""
    o = np.zeros(4)
    lib().orc_time_at_phi(e2, phi, h0, _dp(o))
    return tuple(o)


def u_of_phi(e2: float, phi: float, h0: float = 1e-4) -> float:
    return lib().orc_u_of_phi(e2, phi, h0)


def state_at_phi(e2: float, phi: float, h0: float = 1e-4):
    o = np.zeros(2)
    lib().orc_state_at_phi(e2, phi, h0, _dp(o))
    return o[0], o[1]


def apsis_deflection(e2: float, h0: float = 1e-4) -> float:
    """Delta_a = phi_a - pi/2 on the ray from infinity (e^2 < mu)."""
    return lib().orc_apsis_deflection(e2, h0)


def d_lookup(D: np.ndarray, e2: float, u: float) -> float:
    D = np.ascontiguousarray(D, dtype=np.float64)
    return lib().orc_d_lookup(_dp(D), D.shape[0], e2, u)


def u_lookup(U: np.ndarray, e2: float, phi: float) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_u_lookup(_dp(U), U.shape[1], U.shape[0], e2, phi)


def trace_ray(D, U, pr, delta, alpha, u_ic, u_oc, alpha_valid=True):
    """Algorithm 1 TRACERAY.  Returns dict(delta_p, hits=[(u, angle)], e2)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    o = np.zeros(10)
    lib().orc_trace_ray(_dp(D), D.shape[0], _dp(U), U.shape[1], U.shape[0], pr, delta, alpha,
                        int(alpha_valid), u_ic, u_oc, _dp(o))
    hits = [(o[2 + 2 * k], o[3 + 2 * k]) for k in range(int(o[1]))]
    return {"delta_p": o[0], "hits": hits, "e2": o[6]}


def trace_ray_t(D, DT, U, UT, pr, delta, alpha, u_ic, u_oc, alpha_valid=True):
    """TRACERAY with the retarded times of the hits (camera time minus emission)."""
    arr = [np.ascontiguousarray(a, dtype=np.float64) for a in (D, DT, U, UT)]
    o = np.zeros(10)
    lib().orc_trace_ray2(_dp(arr[0]), _dp(arr[1]), arr[0].shape[0], _dp(arr[2]), _dp(arr[3]),
                         arr[2].shape[1], arr[2].shape[0], pr, delta, alpha, int(alpha_valid), u_ic,
                         u_oc, _dp(o))
    hits = [(o[2 + 2 * k], o[3 + 2 * k], o[8 + k]) for k in range(int(o[1]))]
    return {"delta_p": o[0], "hits": hits, "e2": o[6]}


# --------------------------------------------------------------------------
# Colour (Sec. 3.4.2)
# --------------------------------------------------------------------------

def cmf(lam: float):
    o = np.zeros(3)
    lib().orc_cmf(lam, _dp(o))
    return o


def planck(lam: float, T: float) -> float:
    return lib().orc_planck(lam, T)


def blackbody_xyz(T: float):
    o = np.zeros(3)
    lib().orc_blackbody_xyz(T, _dp(o))
    return o


def xyz_to_rgb_matrix():
    o = np.zeros(9)
    lib().orc_xyz_to_rgb_matrix(_dp(o))
    return o.reshape(3, 3)


def disc_colour_table(n: int = 1024):
    o = np.zeros((n, 3))
    lib().orc_disc_colour_table(n, _dp(o))
    return o


def disc_xyz(table: np.ndarray, T: float):
    """XYZ of the black body at T read from a disc colour table (n, 3) as the
    render reads it (ln Y, X/Y, Z/Y linear in log2 T; 0 below 256 K)."""
    t = np.ascontiguousarray(table, dtype=np.float64)
    o = np.zeros(3)
    lib().orc_disc_xyz(_dp(t), t.shape[0], T, _dp(o))
    return o


def colour_table(nx: int = 64, ny: int = 32, nd: int = 64):
    o = np.zeros((nd, ny, nx, 3))
    if lib().orc_colour_table(nx, ny, nd, _dp(o)):
        raise MemoryError
    return o


def star_xyz(lum: float, temp: float):
    o = (C.c_float * 3)()
    lib().orc_star_xyz(lum, temp, o)
    return np.array(o[:], dtype=np.float32)


# --------------------------------------------------------------------------
# Star cube map (Sec. 3.3.2 "Emitted light")
# --------------------------------------------------------------------------

def cube_levels(N: int) -> int:
    return lib().orc_cube_levels(N)


def cube_level_offset(N: int, L: int) -> int:
    return lib().orc_cube_level_offset(N, L)


def cube_records(N: int) -> int:
    return cube_level_offset(N, cube_levels(N))


def build_cubemap(stars: np.ndarray, N: int, dtype: int = 1) -> np.ndarray:
    """stars: (n, 5) float32 [dir x, y, z, luminosity, temperature K].
    dtype 1 = half, 2 = bfloat16.  Returns uint16 records (n_texels, 4)."""
    stars = np.ascontiguousarray(stars, dtype=np.float32)
    rec = np.zeros((cube_records(N), 4), dtype=np.uint16)
    rc = lib().orc_build_cubemap(stars.ctypes.data_as(C.POINTER(C.c_float)), stars.shape[0], N,
                                 dtype, rec.ctypes.data_as(C.POINTER(C.c_uint16)))
    if rc:
        raise ValueError(f"orc_build_cubemap failed ({rc})")
    return rec


def decode16(h: int, dtype: int) -> float:
    return lib().orc_decode16(int(h), dtype)


def encode16(v: float, dtype: int) -> int:
    return lib().orc_encode16(v, dtype)


# --------------------------------------------------------------------------
# Camera, beam, render
# --------------------------------------------------------------------------

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
    """d may carry "particles" ((n, 3): u1, u2, phi0) and "time" (Appendix B)."""
    x = Disc()
    x.r_in, x.r_out, x.t_peak, x.density = d["r_in"], d["r_out"], d["t_peak"], d["density"]
    x.enabled = int(d.get("enabled", 1))
    parts = d.get("particles")
    if parts is not None and len(parts):
        arr = np.ascontiguousarray(parts, dtype=np.float64).reshape(-1, 3)
        x._keep = arr  # the struct points into it
        x.particles, x.n_particles = _dp(arr), arr.shape[0]
    x.time = float(d.get("time", 0.0))
    return x


def beam(cam: dict, qw: float, qh: float) -> dict:
    """Eq. d, Eq. raybasis and Eq. alpha for screen point (qw, qh)."""
    o = np.zeros(16)
    c = make_camera(cam)
    lib().orc_beam(C.byref(c), qw, qh, _dp(o))
    return {"q": o[0:3], "dcart": o[3:6], "dcam": o[6], "delta": o[7], "ey": o[8:11],
            "ez": o[11:14], "alpha": o[14], "alpha_valid": bool(o[15])}


def disc_doppler(dcam, ucam, e, up, ezz) -> float:
    return lib().orc_disc_doppler(dcam, ucam, e, up, ezz)


def disc_temperature(t_peak, u) -> float:
    return lib().orc_disc_temperature(t_peak, u)


class SceneTables:
    """Stored tables, dequantised to double, that a render reads."""

    def __init__(self, D, U, Ct, disc_ln, cube=None, cube_n=0, cube_dtype=1, DT=None, UT=None):
        self.D = np.ascontiguousarray(D, dtype=np.float64)
        self.U = np.ascontiguousarray(U, dtype=np.float64)
        self.DT = None if DT is None else np.ascontiguousarray(DT, dtype=np.float64)
        self.UT = None if UT is None else np.ascontiguousarray(UT, dtype=np.float64)
        self.C = np.ascontiguousarray(Ct, dtype=np.float64)
        self.disc_ln = np.ascontiguousarray(disc_ln, dtype=np.float64)
        self.cube = None if cube is None else np.ascontiguousarray(cube, dtype=np.uint16)
        self.cube_n = cube_n
        self.cube_dtype = cube_dtype

    def scene(self) -> Scene:
        s = Scene()
        s.D, s.d_n = _dp(self.D), self.D.shape[0]
        s.U, s.u_ne, s.u_nphi = _dp(self.U), self.U.shape[1], self.U.shape[0]
        if self.DT is not None and self.UT is not None:
            s.DT, s.UT = _dp(self.DT), _dp(self.UT)
        s.C = _dp(self.C)
        s.c_nd, s.c_ny, s.c_nx = self.C.shape[0], self.C.shape[1], self.C.shape[2]
        s.disc_ln, s.disc_n = _dp(self.disc_ln), self.disc_ln.shape[0]
        if self.cube is not None:
            s.cube = self.cube.ctypes.data_as(C.POINTER(C.c_uint16))
        s.cube_n, s.cube_dtype = self.cube_n, self.cube_dtype
        return s


def render(cam: dict, disc: dict, tables: SceneTables, exposure_disc=1.0, exposure_stars=0.01,
           y0=0, y1=None, force_level=-1, nthreads=None, debug=False):
    """Per-pixel render of rows [y0, y1).  Returns (rgba (rows, W, 4), dbg or None,
    texels visited)."""
    c = make_camera(cam)
    d = make_disc(disc)
    y1 = cam["height"] if y1 is None else y1
    W = cam["width"]
    out = np.zeros((y1 - y0, W, 4))
    dbg = np.zeros((y1 - y0, W, NDBG)) if debug else None
    tex = C.c_longlong(0)
    s = tables.scene()
    nthreads = nthreads or (os.cpu_count() or 1)
    rc = lib().orc_render(C.byref(c), C.byref(d), exposure_disc, exposure_stars, C.byref(s), y0,
                          y1, force_level, nthreads, _dp(out),
                          _dp(dbg) if dbg is not None else None, C.byref(tex))
    if rc:
        raise ValueError(f"orc_render failed ({rc})")
    return out, dbg, tex.value


def bruteforce_ray(x0, d0, r_in=3.0, r_out=12.0, step=1e-3):
    """Table-free 3D photon orbit; returns dict(dir, captured, hits_u)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    d0 = np.ascontiguousarray(d0, dtype=np.float64)
    o = np.zeros(17)
    lib().orc_bruteforce_ray(_dp(x0), _dp(d0), r_in, r_out, step, _dp(o))
    n = min(int(o[4]), 4)
    return {"dir": o[0:3], "captured": bool(o[3]), "hits_u": list(o[5:5 + n]),
            "hits_t": list(o[9:9 + n]), "hits_phi": list(o[13:13 + n]), "n_crossings": int(o[4])}


# --------------------------------------------------------------------------
# Free-fall camera orbit (Appendix C)
# --------------------------------------------------------------------------

def ellipk(k: float) -> float:
    """Complete elliptic integral of the first kind K(k) (modulus k)."""
    return lib().orc_ellipk(k)


def particle_point(p, t: float, a: float):
    """(u, phi) of point a of linear particle p = (u1, u2, phi0) at time t."""
    u, ph = C.c_double(), C.c_double()
    arr = np.ascontiguousarray(p, dtype=np.float64)
    lib().orc_particle_point(_dp(arr), t, a, C.byref(u), C.byref(ph))
    return u.value, ph.value


def disc_density(particles, rho: float, ht: float, hr: float, hphi: float) -> float:
    arr = np.ascontiguousarray(particles, dtype=np.float64).reshape(-1, 3)
    return lib().orc_disc_density(_dp(arr), arr.shape[0], rho, ht, hr, hphi)


def orbit_init(r0, delta0, v0, chi) -> Orbit:
    o = Orbit()
    if lib().orc_orbit_init(r0, delta0, v0, chi, C.byref(o)):
        raise ValueError("orbit_init: need r0 > 1 and 0 <= v0 < 1")
    return o


def orbit_advance(o: Orbit, dtau: float, n: int = 100) -> Orbit:
    lib().orc_orbit_advance(C.byref(o), dtau, n)
    return o


def orbit_camera(o: Orbit, orient=((1, 0, 0), (0, 1, 0), (0, 0, 1)), fov_y=1.0471975511965976,
                 width=64, height=64) -> dict:
    """Camera dict (as the render takes) of an orbit state; orient rows on the
    boosted (r', chi', psi') axes."""
    oo = np.ascontiguousarray(np.asarray(orient, dtype=np.float64).reshape(9))
    out = np.zeros(15)
    lib().orc_orbit_camera(C.byref(o), _dp(oo), _dp(out))
    return {"r": out[0], "theta": out[1], "phi": out[2], "v": tuple(out[3:6]),
            "orient": tuple(tuple(out[6 + 3 * i:9 + 3 * i]) for i in range(3)),
            "fov_y": fov_y, "width": width, "height": height}
