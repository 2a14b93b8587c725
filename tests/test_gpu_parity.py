"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tables: GPU FP64 quadrature vs the oracle's RK4 tables, <= 1e-6 relative.
Cube map: bit-exact records.  Render: per-stage values and linear RGB on the
same seeded inputs, outside the oracle-derived mask of discontinuities;
full-size workloads on sampled rows; batched and served renders equal to
single renders bit for bit.
"""
import math

import numpy as np
import pytest

from paper_2010_08735_gb300 import synth
from gpu_helpers import (HIT_U_REL, RGB_MAX_REL, RGB_MEAN_REL, TABLE_REL, image_error,
                         ill_conditioned_ok, mask_report, maybe_dump, oracle_mask,
                         star_ill_conditioned)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2010_08735_gb300 import bh  # noqa: E402

MU = 4.0 / 27.0
EXPOSURE_STARS = 0.05


@pytest.fixture(scope="module")
def ctx():
    c = bh.bh_create(0, 0)
    yield c
    bh.bh_destroy(c)


@pytest.fixture(scope="module")
def orc_tables_t(orc):
    """D, U and their regularised-time channels DT, UT."""
    return orc.tables_exact_t(512, 64, 32, 1e-3)


@pytest.fixture(scope="module")
def orc_tables(orc_tables_t):
    return orc_tables_t[:2]


@pytest.fixture(scope="module")
def orc_colour(orc):
    return orc.colour_table(64, 32, 64), orc.disc_colour_table(1024)


@pytest.fixture(scope="module")
def gpu_tables(ctx):
    t = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F32)
    yield t
    bh.bh_tables_free(t)


@pytest.fixture(scope="module")
def uploaded_tables(ctx, orc_tables):
    D, U = orc_tables
    t = bh.bh_tables_upload(ctx, D, U, bh.BH_F32)
    yield t
    bh.bh_tables_free(t)


# ---------------------------------------------------------------------------
# tables (a10, a11, a13)
# ---------------------------------------------------------------------------

def test_tables_match_oracle(gpu_tables, orc_tables):
    Dg, Ug = bh.bh_tables_copy_out(gpu_tables, 512, 64, 32)
    Do, Uo = orc_tables
    errD = np.abs(Dg - Do) / (np.abs(Do) + 1e-3)
    assert errD.max() <= TABLE_REL, np.unravel_index(errD.argmax(), errD.shape)
    errU = np.abs(Ug - Uo) / (np.abs(Uo) + 1e-6)
    assert errU.max() <= TABLE_REL, np.unravel_index(errU.argmax(), errU.shape)


def test_time_tables_match_oracle(gpu_tables, orc_tables_t):
    """Regularised-time channels (Algorithm 1 stores t beside Delta and u)."""
    DTg, UTg = bh.bh_tables_copy_time(gpu_tables, 512, 64, 32)
    DTo, UTo = orc_tables_t[2:]
    errD = np.abs(DTg - DTo) / (np.abs(DTo) + 1e-3)
    assert errD.max() <= TABLE_REL, np.unravel_index(errD.argmax(), errD.shape)
    errU = np.abs(UTg - UTo) / (np.abs(UTo) + 1e-3)
    assert errU.max() <= TABLE_REL, np.unravel_index(errU.argmax(), errU.shape)


@pytest.mark.parametrize("dn,une,unphi", [(66, 10, 6), (128, 16, 16), (4, 2, 2)])
def test_tables_small_and_ragged(ctx, orc, dn, une, unphi):
    t = bh.bh_precompute_tables(ctx, dn, une, unphi, bh.BH_F16)
    try:
        Dg, Ug = bh.bh_tables_copy_out(t, dn, une, unphi)
        DTg, UTg = bh.bh_tables_copy_time(t, dn, une, unphi)
    finally:
        bh.bh_tables_free(t)
    Do, Uo, DTo, UTo = orc.tables_exact_t(dn, une, unphi, 1e-3)
    assert (np.abs(Dg - Do) / (np.abs(Do) + 1e-3)).max() <= TABLE_REL
    assert (np.abs(Ug - Uo) / (np.abs(Uo) + 1e-6)).max() <= TABLE_REL
    assert (np.abs(DTg - DTo) / (np.abs(DTo) + 1e-3)).max() <= TABLE_REL
    assert (np.abs(UTg - UTo) / (np.abs(UTo) + 1e-3)).max() <= TABLE_REL


def test_uploaded_tables_time_channel(ctx, orc_tables_t):
    """Uploaded tables carry NaN time channels until bh_tables_upload_time."""
    D, U, DT, UT = orc_tables_t
    t = bh.bh_tables_upload(ctx, D, U, bh.BH_F16)
    try:
        DTg, UTg = bh.bh_tables_copy_time(t, 512, 64, 32)
        assert np.isnan(DTg).all() and np.isnan(UTg).all()
        bh.bh_tables_upload_time(t, DT, UT)
        DTg, UTg = bh.bh_tables_copy_time(t, 512, 64, 32)
        assert np.array_equal(DTg, DT) and np.array_equal(UTg, UT)
    finally:
        bh.bh_tables_free(t)


def test_colour_tables_match_oracle(gpu_tables, orc_colour):
    """C(xy, D) and the disc black-body table: both computed in FP64 on the
    GPU and stored as FP32, so each value is the oracle's to within the FP32
    rounding of its storage: 2^-24 relative, or, for the faint corners of C
    below FP32's normal range (1.18e-38), that range's absolute spacing."""
    Cg, dg = bh.bh_tables_copy_colour(gpu_tables)
    Co, do = orc_colour
    tiny = float(np.finfo(np.float32).tiny)
    for name, g, o in (("C", Cg[..., :3], Co), ("disc", dg[:, :3], do)):
        err = np.abs(g.astype(np.float64) - o)
        bound = 2.0 ** -24 * np.abs(o) * (1 + 1e-6) + tiny
        normal = np.abs(o) >= tiny
        print(f"{name} table: max relative difference {(err[normal] / np.abs(o[normal])).max():.3e} "
              f"over {normal.sum()} normal values, {(~normal).sum()} below FP32's normal range")
        assert np.all(err <= bound), name


def test_invalid_arguments(ctx, gpu_tables):
    out = torch.zeros((4, 4, 4), device="cuda")
    sh = bh.make_shading()
    bad = [synth.camera(1.0, 80, width=4, height=4), synth.camera(10, 80, v=(0.6, 0.6, 0.6), width=4, height=4),
           dict(synth.camera(10, 80, width=4, height=4), orient=((1, 0, 0), (1, 0, 0), (0, 0, 1))),
           synth.camera(10, 80, width=0, height=4)]
    for cam in bad:
        with pytest.raises(bh.BhError) as ei:
            bh.bh_render(ctx, gpu_tables, None, cam, synth.disc(), sh, out)
        assert ei.value.status == bh.BH_ERR_INVALID_ARG
    with pytest.raises(bh.BhError):
        bh.bh_render(ctx, gpu_tables, None, synth.camera(10, 80, width=4, height=4),
                     synth.disc(2.0, 12.0), sh, out)
    with pytest.raises(bh.BhError):
        bh.bh_precompute_tables(ctx, 511, 64, 32)


# ---------------------------------------------------------------------------
# cube map (a12)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,N,dtype", [(1000, 2048, 1), (20000, 64, 1), (5000, 128, 2), (0, 8, 1),
                                       (300000, 256, 1)])
def test_cubemap_bit_exact(ctx, orc, n, N, dtype):
    st = synth.stars(n, seed=11)
    c = bh.bh_build_star_cubemap(ctx, st, N, dtype)
    try:
        rec = bh.bh_cubemap_copy_out(c, N)
    finally:
        bh.bh_cubemap_free(c)
    ref = orc.build_cubemap(st, N, dtype)
    diff = np.any(rec != ref, axis=1)
    assert diff.sum() == 0, (diff.sum(), np.flatnonzero(diff)[:5])


def test_cubemap_from_device_stars(ctx, orc):
    st = synth.stars(4000, seed=12)
    dst = torch.from_numpy(st).cuda()
    c = bh.bh_build_star_cubemap(ctx, dst, 128, 1)
    try:
        rec = bh.bh_cubemap_copy_out(c, 128)
    finally:
        bh.bh_cubemap_free(c)
    assert np.array_equal(rec, orc.build_cubemap(st, 128, 1))


# ---------------------------------------------------------------------------
# render (a1..a9)
# ---------------------------------------------------------------------------

def gpu_render(ctx, tables, cube, cam, disc, debug=True, exposure_stars=EXPOSURE_STARS):
    W, H = cam["width"], cam["height"]
    out = torch.zeros((H, W, 4), device="cuda")
    sh = bh.make_shading(1.0, exposure_stars)
    if debug:
        dbg = torch.zeros((H, W, bh.NDBG), device="cuda")
        bh.bh_render_debug(ctx, tables, cube, cam, disc, sh, out, dbg)
        torch.cuda.synchronize()
        # the debug render checks every table, cube-map and occupancy index
        assert bh.bh_check_status(ctx) == bh.BH_OK
        return out.cpu().numpy(), dbg.cpu().numpy()
    bh.bh_render(ctx, tables, cube, cam, disc, sh, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), None


def orc_scene(orc, orc_tables, orc_colour, cube_rec, N, dtype):
    D, U = orc_tables
    Ct, dl = orc_colour
    # the renderer reads FP32-stored tables
    return orc.SceneTables(D.astype(np.float32), U.astype(np.float32), Ct.astype(np.float32),
                           dl.astype(np.float32), cube_rec, N, dtype)


@pytest.fixture(scope="module")
def static_scene(ctx, orc, orc_tables, orc_colour):
    wk = synth.WORKLOADS["static_256"]
    st = synth.stars(wk["n_stars"], wk["star_seed"])
    N = wk["cube_n"]
    cube = bh.bh_build_star_cubemap(ctx, st, N, 1)
    rec = orc.build_cubemap(st, N, 1)
    yield cube, orc_scene(orc, orc_tables, orc_colour, rec, N, 1)
    bh.bh_cubemap_free(cube)


def compare_render(orc, ctx, tables, cube, scene, cam, disc, y0=0, y1=None, name="render"):
    og, gd = gpu_render(ctx, tables, cube, cam, disc)
    y1 = cam["height"] if y1 is None else y1
    oo, od, _ = orc.render(cam, disc, scene, exposure_stars=EXPOSURE_STARS, y0=y0, y1=y1,
                           debug=True)
    og, gd = og[y0:y1], gd[y0:y1]
    mask = oracle_mask(od)
    maybe_dump(name, og=og, gd=gd, oo=oo, od=od, mask=mask)
    return og, gd, oo, od, mask


def check_stages(gd, od, mask):
    cap_o = ~np.isfinite(od[..., 2])
    cap_g = ~np.isfinite(gd[..., 2])
    assert np.array_equal(cap_o[~mask], cap_g[~mask])
    ok = ~mask & ~cap_o
    # e^2 and delta (FP32 vs FP64)
    assert np.allclose(gd[..., 1][ok], od[..., 1][ok], atol=2e-5)
    # escape angle, away from the photon sphere where it is ill-conditioned
    far = ok & (np.abs(od[..., 0] / MU - 1) > 1e-2)
    if far.any():
        dd = np.abs(np.angle(np.exp(1j * (gd[..., 2][far] - od[..., 2][far]))))
        assert dd.max() < 1e-3, dd.max()
    # disc hits: same count and radius within 1e-3 relative
    same = ~mask & (gd[..., 3] == od[..., 3])
    nhit = (~mask & (gd[..., 3] != od[..., 3])).sum()
    print(f"HITCOUNT differing on {nhit} of {(~mask).sum()} unmasked pixels")
    assert nhit <= 0.001 * (~mask).sum()
    for k, ch in ((1, 4), (2, 5)):
        sel = same & (od[..., 3] >= k)
        if sel.any():
            rel = np.abs(gd[..., ch][sel] - od[..., ch][sel]) / od[..., ch][sel]
            assert rel.max() <= HIT_U_REL, rel.max()
    # mip level and face agree outside the mask
    has = ~mask & (od[..., 6] >= 0)
    if has.any():
        assert (gd[..., 6][has] != od[..., 6][has]).mean() < 1e-3
        assert (gd[..., 7][has] != od[..., 7][has]).mean() < 1e-3


def check_rgb(og, oo, od, mask, cam, name="render"):
    mask_report(name, od, oo, cam)
    ill = star_ill_conditioned(od, oo, cam)
    mean, mx, rel = image_error(og, oo, mask | ill)
    assert mean <= RGB_MEAN_REL and mx <= RGB_MAX_REL, (mean, mx)
    assert ill.mean() < 0.10
    assert ill_conditioned_ok(rel, od, oo, cam, mask)


def test_render_static_256(ctx, orc, gpu_tables, static_scene):
    cube, scene = static_scene
    wk = synth.WORKLOADS["static_256"]
    og, gd, oo, od, mask = compare_render(orc, ctx, gpu_tables, cube, scene, wk["camera"], wk["disc"],
                                          name="static_256")
    assert mask.mean() < 0.2
    check_stages(gd, od, mask)
    check_rgb(og, oo, od, mask, wk["camera"], "static_256")


def test_render_uploaded_tables_static_256(ctx, orc, uploaded_tables, static_scene):
    cube, scene = static_scene
    wk = synth.WORKLOADS["static_256"]
    og, gd, oo, od, mask = compare_render(orc, ctx, uploaded_tables, cube, scene, wk["camera"],
                                          wk["disc"], name="static_256_uploaded")
    check_stages(gd, od, mask)
    check_rgb(og, oo, od, mask, wk["camera"], "static_256_uploaded")


ANIM_CAMS = [
    (synth.WORKLOADS["static_256"]["camera"], synth.WORKLOADS["static_256"]["disc"], 250.0),
    (synth.camera(6.0, 85.0, v=(0.0, 0.0, 0.5), width=192, height=108), synth.disc(3.0, 12.0), 1.0e4),
    (synth.camera(25.0, 60.0, phi_deg=40.0, v=(0.2, -0.3, 0.1), width=97, height=61), synth.disc(3.0, 20.0), 37.5),
]


@pytest.mark.parametrize("k", range(len(ANIM_CAMS)))
def test_render_animated_disc(ctx, orc, orc_tables_t, orc_colour, gpu_tables, static_scene, k):
    """Animated disc (Appendix B): per-hit densities at the retarded times
    (debug channels 18, 19) and the image, against the oracle."""
    cam, disc0, time = ANIM_CAMS[k]
    cube, scene0 = static_scene
    D, U, DT, UT = orc_tables_t
    parts = synth.disc_particles(16, 5, disc0["r_in"], disc0["r_out"])
    f32 = lambda a: a.astype(np.float32)
    scene = orc.SceneTables(f32(D), f32(U), scene0.C, scene0.disc_ln, scene0.cube, scene0.cube_n,
                            scene0.cube_dtype, DT=f32(DT), UT=f32(UT))
    ph = bh.bh_disc_particles_create(ctx, parts)
    try:
        disc = dict(disc0, particles=parts, particles_handle=ph, time=time)
        og, gd, oo, od, mask = compare_render(orc, ctx, gpu_tables, cube, scene, cam, disc,
                                              name=f"anim_{cam['width']}x{cam['height']}")
    finally:
        bh.bh_disc_particles_free(ph)
    check_stages(gd, od, mask)
    same = ~mask & (gd[..., 3] == od[..., 3])
    n = 0
    for h in (0, 1):
        sel = same & (od[..., 3] >= h + 1)
        if sel.any():
            n += sel.sum()
            err = np.abs(gd[..., 18 + h][sel] - od[..., 25 + h][sel])
            assert err.max() <= 2e-3, (h, err.max())
    assert n > 0
    dens = od[..., 25][od[..., 3] >= 1]
    assert dens.std() > 0.1 and (dens < 1).mean() > 0.5  # the density varies, mostly unclamped
    check_rgb(og, oo, od, mask, cam, "animated")


def test_disc_particles_invalid(ctx):
    good = synth.disc_particles(4, 5)
    for bad in (good[:0], np.vstack([good] * 65), np.array([[0.2, 0.1, 0.0]]), np.array([[0.1, 0.4, 0.0]]),
                np.array([[0.0, 0.1, 0.0]]), np.array([[0.1, 0.1, np.nan]])):
        with pytest.raises(bh.BhError):
            bh.bh_disc_particles_create(ctx, bad)


DELAY_CAMS = [
    (synth.WORKLOADS["static_256"]["camera"], synth.WORKLOADS["static_256"]["disc"]),
    (synth.camera(25.0, 60.0, phi_deg=40.0, v=(0.2, -0.3, 0.1), width=97, height=61), synth.disc(3.0, 20.0)),
    (synth.camera(3.2, 89.0, v=(-0.9, 0.0, 0.0), width=96, height=54), synth.disc(3.0, 20.0)),
]


@pytest.mark.parametrize("uploaded", [False, True])
@pytest.mark.parametrize("k", range(len(DELAY_CAMS)))
def test_render_hit_delays(ctx, orc, orc_tables_t, orc_colour, gpu_tables, uploaded, k):
    """Retarded-time delays of the disc hits (debug channels 16, 17) against
    the oracle's TRACERAY with the time channels stored in FP32 like the GPU's."""
    cam, disc = DELAY_CAMS[k]
    D, U, DT, UT = orc_tables_t
    Ct, dl = orc_colour
    f32 = lambda a: a.astype(np.float32)
    scene = orc.SceneTables(f32(D), f32(U), f32(Ct), f32(dl), DT=f32(DT), UT=f32(UT))
    t = gpu_tables
    if uploaded:
        t = bh.bh_tables_upload(ctx, D, U, bh.BH_F32)
        bh.bh_tables_upload_time(t, DT, UT)
    try:
        _, gd = gpu_render(ctx, t, None, cam, disc)
    finally:
        if uploaded:
            bh.bh_tables_free(t)
    _, od, _ = orc.render(cam, disc, scene, exposure_stars=EXPOSURE_STARS, debug=True)
    mask = oracle_mask(od)
    same = ~mask & (gd[..., 3] == od[..., 3])
    nsel = 0
    for h in (0, 1):
        sel = same & (od[..., 3] >= h + 1)
        if not sel.any():
            continue
        nsel += sel.sum()
        g, o = gd[..., 16 + h][sel], od[..., 23 + h][sel]
        # light leaves the disc before it reaches the camera
        assert (o > 0).all() and (g > 0).all()
        rel = np.abs(g - o) / np.maximum(np.abs(o), 1.0)
        assert rel.max() <= HIT_U_REL, (h, rel.max())
    assert nsel > 0
    # no hit: zero delays
    none = gd[..., 3] == 0
    assert (gd[..., 16][none] == 0).all() and (gd[..., 17][none] == 0).all()


@pytest.mark.parametrize("cam", [
    synth.camera(6.0, 85.0, v=(0.0, 0.0, 0.5), width=192, height=108),
    synth.camera(3.2, 89.0, v=(-0.9, 0.0, 0.0), width=96, height=54),
    synth.camera(25.0, 60.0, phi_deg=40.0, v=(0.2, -0.3, 0.1), width=97, height=61),  # ragged
    synth.camera(1.3, 30.0, v=(0.0, 0.4, 0.0), width=64, height=64),  # inside the photon sphere
    synth.camera(8.0, 10.0, width=3, height=1),
    synth.camera(8.0, 10.0, width=1, height=1),
    synth.camera(6.0, 90.0, width=65, height=49),  # in the disc plane, inside the disc; odd sizes
    synth.camera(1.02, 60.0, width=48, height=32),  # just outside the horizon
    synth.camera(10.0, 80.0, v=(0.0, 0.0, 0.99), width=64, height=48),  # v = 0.99c
])
def test_render_configs_small(ctx, orc, gpu_tables, static_scene, cam):
    cube, scene = static_scene
    disc = synth.disc(3.0, 20.0)
    og, gd, oo, od, mask = compare_render(orc, ctx, gpu_tables, cube, scene, cam, disc,
                                          name=f"small_{cam['width']}x{cam['height']}_r{cam['r']}")
    check_stages(gd, od, mask)
    check_rgb(og, oo, od, mask, cam, "small")


def test_empty_star_field_equals_no_cube_map(ctx, gpu_tables):
    """A cube map built from no stars adds no light: the frame equals the one
    rendered without a cube map, bit for bit, in the timed and debug forms."""
    cube = bh.bh_build_star_cubemap(ctx, np.zeros((0, 5), dtype=np.float32), 256, 1)
    try:
        cam = synth.camera(6.0, 85.0, v=(0.0, 0.0, 0.5), width=96, height=54)
        disc = synth.disc(3.0, 20.0)
        with_cube, _ = gpu_render(ctx, gpu_tables, cube, cam, disc, debug=False)
        without, _ = gpu_render(ctx, gpu_tables, None, cam, disc, debug=False)
        assert np.array_equal(with_cube, without)
        dbg_cube, _ = gpu_render(ctx, gpu_tables, cube, cam, disc)
        assert np.array_equal(dbg_cube, without)
    finally:
        bh.bh_cubemap_free(cube)


def test_star_centroids_sparse_field(ctx, orc, orc_tables, orc_colour, gpu_tables):
    """Intensity-weighted centroids of isolated star images agree within 0.05 px."""
    st = synth.stars(100, seed=3)
    N = 2048
    cube = bh.bh_build_star_cubemap(ctx, st, N, 1)
    try:
        scene = orc_scene(orc, orc_tables, orc_colour, orc.build_cubemap(st, N, 1), N, 1)
        cam = synth.camera(12.0, 70.0, width=256, height=256, fov_deg=90.0)
        disc = synth.disc(enabled=False)
        _, gd = gpu_render(ctx, gpu_tables, cube, cam, disc)
        _, od, _ = orc.render(cam, disc, scene, exposure_stars=EXPOSURE_STARS, debug=True)
    finally:
        bh.bh_cubemap_free(cube)
    Yg, Yo = gd[..., 11], od[..., 11]
    lit = Yo > 0
    from scipy import ndimage
    lab, nl = ndimage.label(lit)
    checked = 0
    for k in range(1, nl + 1):
        sel = lab == k
        if sel.sum() > 16:
            continue  # merged or lensed into an arc: not an isolated star image
        jj, ii = np.nonzero(sel)
        wo, wg = Yo[sel], Yg[sel]
        if wg.sum() <= 0:
            continue
        co = np.array([(wo * ii).sum(), (wo * jj).sum()]) / wo.sum()
        cg = np.array([(wg * ii).sum(), (wg * jj).sum()]) / wg.sum()
        assert np.abs(co - cg).max() <= 0.05, (k, co, cg)
        checked += 1
    assert checked >= 10


def test_batch_equals_single(ctx, gpu_tables, static_scene):
    cube, _ = static_scene
    cams = synth.batch_cameras(6, seed=1, resolutions=((64, 48), (33, 17), (128, 72)))
    disc = synth.disc()
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    outs = [torch.zeros((c["height"], c["width"], 4), device="cuda") for c in cams]
    bh.bh_render_batch(ctx, gpu_tables, cube, cams, disc, sh, outs)
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        single = torch.zeros_like(o)
        bh.bh_render(ctx, gpu_tables, cube, c, disc, sh, single)
        torch.cuda.synchronize()
        assert torch.equal(single, o)


def test_autotune_every_candidate_same_image(gpu_tables, static_scene):
    """The autotuner launches every candidate launch shape; the image does not
    depend on the shape, and batched renders stay equal to single ones."""
    cube, _ = static_scene
    c2 = bh.bh_create(0, 0)
    try:
        cams = synth.batch_cameras(4, seed=1, resolutions=((64, 48), (33, 17), (128, 72)))
        disc = synth.disc()
        sh = bh.make_shading(1.0, EXPOSURE_STARS)
        before = []
        for c in cams:
            o = torch.zeros((c["height"], c["width"], 4), device="cuda")
            bh.bh_render(c2, gpu_tables, cube, c, disc, sh, o)
            before.append(o)
        outs = [torch.zeros_like(o) for o in before]
        choice = bh.bh_autotune_batch(c2, gpu_tables, cube, cams, disc, sh, outs)
        assert choice >= 0
        outs = [torch.zeros_like(o) for o in before]
        bh.bh_render_batch(c2, gpu_tables, cube, cams, disc, sh, outs)
        torch.cuda.synchronize()
        for b, o in zip(before, outs):
            assert torch.equal(b, o)
    finally:
        bh.bh_destroy(c2)


def test_checkpoints_round_trip(ctx, gpu_tables, static_scene, tmp_path):
    """Tables and cube maps saved to disk load back equal, render the same
    image, and damaged files are refused before anything is allocated."""
    cube, _ = static_scene
    tp, cp = tmp_path / "tables.bht", tmp_path / "cube.bhc"
    bh.bh_tables_save(gpu_tables, tp)
    bh.bh_cubemap_save(cube, cp)
    t2 = bh.bh_tables_load(ctx, tp)
    c2 = bh.bh_cubemap_load(ctx, cp)
    try:
        for a, b in zip(bh.bh_tables_copy_out(gpu_tables, 512, 64, 32) + bh.bh_tables_copy_time(gpu_tables, 512, 64, 32),
                        bh.bh_tables_copy_out(t2, 512, 64, 32) + bh.bh_tables_copy_time(t2, 512, 64, 32)):
            assert np.array_equal(a, b)
        for a, b in zip(bh.bh_tables_copy_colour(gpu_tables), bh.bh_tables_copy_colour(t2)):
            assert np.array_equal(a, b)
        assert np.array_equal(bh.bh_cubemap_copy_out(cube, 2048), bh.bh_cubemap_copy_out(c2, 2048))
        cam = synth.camera(10.0, 80.0, width=96, height=64)
        sh = bh.make_shading(1.0, EXPOSURE_STARS)
        a = torch.zeros((64, 96, 4), device="cuda")
        b = torch.zeros_like(a)
        bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, a)
        bh.bh_render(ctx, t2, c2, cam, synth.disc(), sh, b)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    finally:
        bh.bh_tables_free(t2)
        bh.bh_cubemap_free(c2)
    raw = bytearray(tp.read_bytes())
    bad = tmp_path / "bad.bht"
    for damage in ("flip", "truncate", "magic"):
        d = bytearray(raw)
        if damage == "flip":
            d[len(d) // 2] ^= 0x40
        elif damage == "truncate":
            d = d[:-100]
        else:
            d[0:8] = b"NOTTABLE"
        bad.write_bytes(bytes(d))
        with pytest.raises(bh.BhError):
            bh.bh_tables_load(ctx, bad)
    with pytest.raises(bh.BhError):
        bh.bh_cubemap_load(ctx, tp)  # a tables file is not a cube map
    with pytest.raises(bh.BhError):
        bh.bh_tables_load(ctx, tmp_path / "missing.bht")


def test_render_to_host_equals_device(ctx, gpu_tables, static_scene):
    cube, _ = static_scene
    cam = synth.camera(10.0, 80.0, width=80, height=40)
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    dev = torch.zeros((40, 80, 4), device="cuda")
    bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, dev)
    host = np.zeros((40, 80, 4), dtype=np.float32)  # pageable: rendered on the device, then copied
    bh.bh_render_to_host(ctx, gpu_tables, cube, cam, synth.disc(), sh, host)
    assert np.array_equal(host, dev.cpu().numpy())
    pinned = torch.zeros((40, 80, 4), dtype=torch.float32).pin_memory()  # written by the kernel directly
    bh.bh_render_to_host(ctx, gpu_tables, cube, cam, synth.disc(), sh, pinned)
    assert torch.equal(pinned, dev.cpu())


@pytest.mark.parametrize("W,H", [(80, 40), (97, 61), (1920, 1080)])
def test_render_to_host_rgb_equals_device(ctx, gpu_tables, static_scene, W, H):
    """Packed linear RGB on the host equals the RGB of the device frame, bit for
    bit: widths divisible by 4 take the staged 16-byte-chunk stores, others the
    per-pixel ones; pinned buffers are written by the kernel, pageable ones
    receive a copy."""
    cube, _ = static_scene
    cam = synth.camera(10.0, 80.0, width=W, height=H)
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    dev = torch.zeros((H, W, 4), device="cuda")
    bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, dev)
    ref = dev.cpu().numpy()[..., :3]
    pinned = torch.full((H, W, 3), -1.0, dtype=torch.float32).pin_memory()
    bh.bh_render_to_host_rgb(ctx, gpu_tables, cube, cam, synth.disc(), sh, pinned)
    assert np.array_equal(pinned.numpy(), ref)
    pageable = np.full((H, W, 3), -1.0, dtype=np.float32)
    bh.bh_render_to_host_rgb(ctx, gpu_tables, cube, cam, synth.disc(), sh, pageable)
    assert np.array_equal(pageable, ref)


def test_host_link_measurement():
    """The device-to-host bandwidth measurement returns plausible rates for
    both paths and rejects sizes below one 16-byte chunk."""
    r = bh.bh_measure_host_link(0, 1 << 24)
    for k in ("copy_engine_gbs", "kernel_stores_gbs"):
        assert 1.0 < r[k] < 5000.0, r
    with pytest.raises(bh.BhError):
        bh.bh_measure_host_link(0, 8)


def test_render_to_host_async_frames_in_flight(ctx, gpu_tables, static_scene):
    """Two frames in flight: a sequence of frames of changing camera, sizes and
    both layouts, each enqueued before the previous one is waited for, lands
    in host memory equal to the device render of the same camera; tickets
    count up; a ticket never issued and a pageable buffer are rejected."""
    cube, _ = static_scene
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    frames = []
    for k, (W, H, rgb) in enumerate([(80, 40, True), (96, 54, True), (97, 61, False), (80, 40, True),
                                     (160, 90, True), (64, 48, False), (80, 40, True)]):
        cam = synth.camera(10.0 + 0.5 * k, 80.0 - 2.0 * k, width=W, height=H)
        dev = torch.zeros((H, W, 4), device="cuda")
        bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, dev)
        torch.cuda.synchronize()
        ref = dev.cpu().numpy()
        frames.append((cam, rgb, ref[..., :3] if rgb else ref))
    hosts = [torch.full((90, 160, 4), -1.0, dtype=torch.float32).pin_memory() for _ in range(2)]
    prev, got = None, []
    for k, (cam, rgb, ref) in enumerate(frames):
        ch = 3 if rgb else 4
        buf = hosts[k & 1].view(-1)[:cam["height"] * cam["width"] * ch].view(cam["height"], cam["width"], ch)
        buf.fill_(-1.0)
        tk = bh.bh_render_to_host_async(ctx, gpu_tables, cube, cam, synth.disc(), sh, buf, rgb)
        if prev is not None:
            assert tk == prev[0] + 1
            bh.bh_host_wait(ctx, prev[0])
            got.append(prev[1].numpy().copy())
        prev = (tk, buf)
    bh.bh_host_wait(ctx, prev[0])
    got.append(prev[1].numpy().copy())
    for (cam, rgb, ref), img in zip(frames, got):
        assert np.array_equal(img, ref)
    with pytest.raises(bh.BhError):
        bh.bh_host_wait(ctx, prev[0] + 1)
    cam = frames[0][0]
    pageable = torch.zeros((cam["height"], cam["width"], 3), dtype=torch.float32)
    with pytest.raises(bh.BhError):
        bh.bh_render_to_host_async(ctx, gpu_tables, cube, cam, synth.disc(), sh, pageable, True)


def test_serve_results_equal_alone(ctx, gpu_tables, static_scene):
    """Continuous batching: frames submitted while others are in flight come
    out equal to the same frame rendered alone."""
    cube, _ = static_scene
    cams = synth.batch_cameras(12, seed=7, resolutions=((64, 48), (96, 54)))
    disc = synth.disc()
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    outs = [torch.zeros((c["height"], c["width"], 4), device="cuda") for c in cams]
    tickets = []
    for v, (c, o) in enumerate(zip(cams, outs)):
        st, t = bh.bh_serve_submit(ctx, gpu_tables, cube, v, c, disc, sh, o)
        assert st == bh.BH_OK
        tickets.append(t)
    lat = []
    for t in tickets:
        st, ms = bh.bh_serve_poll(ctx, t, 5_000_000)
        assert st == bh.BH_OK
        lat.append(ms)
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        single = torch.zeros_like(o)
        bh.bh_render(ctx, gpu_tables, cube, c, disc, sh, single)
        torch.cuda.synchronize()
        assert torch.equal(single, o)
    assert all(x >= 0 for x in lat)


def test_serve_admission(ctx, gpu_tables, static_scene):
    """A frame larger than the context's whole memory budget is refused."""
    cube, _ = static_scene
    c2 = bh.bh_create(0, 64 * 48 * 16)  # room for one 64x48 frame
    try:
        sh = bh.make_shading()
        small = torch.zeros((48, 64, 4), device="cuda")
        big = torch.zeros((64, 64, 4), device="cuda")
        st, _ = bh.bh_serve_submit(c2, gpu_tables, cube, 0, synth.camera(10.0, 80.0, width=64, height=64),
                                   synth.disc(), sh, big)
        assert st == bh.BH_ERR_BUSY
        st, t0 = bh.bh_serve_submit(c2, gpu_tables, cube, 1, synth.camera(10.0, 80.0, width=64, height=48),
                                    synth.disc(), sh, small)
        assert st == bh.BH_OK
        assert bh.bh_serve_poll(c2, t0, 5_000_000)[0] == bh.BH_OK
    finally:
        torch.cuda.synchronize()
        bh.bh_destroy(c2)


# ---------------------------------------------------------------------------
# full-size workloads, sampled rows
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,rows", [("orbit_1080p", (520, 560)), ("infall_4k", (1000, 1016))])
def test_full_size_sampled_rows(ctx, orc, orc_tables, orc_colour, gpu_tables, name, rows):
    wk = synth.WORKLOADS[name]
    st = synth.stars(wk["n_stars"], wk["star_seed"])
    N = wk["cube_n"]
    dt = 1 if wk["cube_dtype"] == "f16" else 2
    cube = bh.bh_build_star_cubemap(ctx, st, N, dt)
    try:
        rec = orc.build_cubemap(st, N, dt)
        # the full cube map of the workload (1M stars at 2048^2 FP16, 4M at
        # 4096^2 BF16), record for record: integer work, exact equality
        assert np.array_equal(bh.bh_cubemap_copy_out(cube, N), rec)
        scene = orc_scene(orc, orc_tables, orc_colour, rec, N, dt)
        og, gd, oo, od, mask = compare_render(orc, ctx, gpu_tables, cube, scene, wk["camera"],
                                              wk["disc"], y0=rows[0], y1=rows[1], name=name)
    finally:
        bh.bh_cubemap_free(cube)
    check_stages(gd, od, mask)
    check_rgb(og, oo, od, mask, wk["camera"], name)


@pytest.mark.parametrize("name", ["orbit_1080p", "infall_4k"])
def test_timed_kernel_equals_checked_render_full_size(gpu_tables, name):
    """The plain kernel, in the launch shape the benchmark times (autotuned on
    the frame), renders every pixel of the full-size frame exactly as the
    checked debug render that the sampled-row and small-image tests compare
    with the oracle."""
    wk = synth.WORKLOADS[name]
    cam, disc = wk["camera"], wk["disc"]
    W, H = cam["width"], cam["height"]
    c2 = bh.bh_create(0, 0)
    cube = bh.bh_build_star_cubemap(c2, synth.stars(wk["n_stars"], wk["star_seed"]), wk["cube_n"],
                                    bh.BH_F16 if wk["cube_dtype"] == "f16" else bh.BH_BF16)
    try:
        sh = bh.make_shading(1.0, 0.01)
        plain = torch.zeros((H, W, 4), device="cuda")
        bh.bh_autotune_batch(c2, gpu_tables, cube, [cam], disc, sh, [plain])
        plain.zero_()
        bh.bh_render(c2, gpu_tables, cube, cam, disc, sh, plain)
        dbg_out = torch.zeros_like(plain)
        dbg = torch.zeros((H, W, bh.NDBG), device="cuda")
        bh.bh_render_debug(c2, gpu_tables, cube, cam, disc, sh, dbg_out, dbg)
        torch.cuda.synchronize()
        assert bh.bh_check_status(c2) == bh.BH_OK
        del dbg
        assert torch.equal(plain, dbg_out)
    finally:
        bh.bh_cubemap_free(cube)
        bh.bh_destroy(c2)


def test_timed_animated_kernel_equals_checked_render_full_size(gpu_tables):
    """The animated-disc kernel the benchmark times (16 linear particles,
    Appendix B) renders every pixel of the 1080p frame exactly as the checked
    debug render -- which test_render_animated_disc compares with the oracle --
    at two frame times."""
    wk = synth.WORKLOADS["orbit_1080p"]
    cam, disc0 = wk["camera"], wk["disc"]
    W, H = cam["width"], cam["height"]
    c2 = bh.bh_create(0, 0)
    cube = bh.bh_build_star_cubemap(c2, synth.stars(wk["n_stars"], wk["star_seed"]), wk["cube_n"], bh.BH_F16)
    ph = bh.bh_disc_particles_create(c2, synth.disc_particles(16, 5, disc0["r_in"], disc0["r_out"]))
    try:
        sh = bh.make_shading(1.0, 0.01)
        plain = torch.zeros((H, W, 4), device="cuda")
        bh.bh_autotune_batch(c2, gpu_tables, cube, [cam], disc0, sh, [plain])
        dbg_out = torch.zeros_like(plain)
        dbg = torch.zeros((H, W, bh.NDBG), device="cuda")
        for t in (3.0, 1234.5):
            disc = dict(disc0, particles_handle=ph, time=t)
            plain.zero_()
            bh.bh_render(c2, gpu_tables, cube, cam, disc, sh, plain)
            bh.bh_render_debug(c2, gpu_tables, cube, cam, disc, sh, dbg_out, dbg)
            torch.cuda.synchronize()
            assert bh.bh_check_status(c2) == bh.BH_OK
            assert torch.equal(plain, dbg_out), t
            dens = dbg[..., 18][dbg[..., 3] >= 1]
            assert dens.numel() > 0 and float(dens.std()) > 0.05  # particles really shade the frame
    finally:
        bh.bh_disc_particles_free(ph)
        bh.bh_cubemap_free(cube)
        bh.bh_destroy(c2)


@pytest.mark.parametrize("cam", [synth.WORKLOADS["static_256"]["camera"],
                                 synth.camera(3.2, 89.0, v=(-0.9, 0.0, 0.0), width=96, height=54)])
def test_render_f16_tables(ctx, orc, orc_tables, orc_colour, static_scene, cam):
    """The FP16 table path (D read through the read-only path, U staged in shared
    memory as halves) against the oracle reading the same FP16-rounded tables."""
    cube, scene32 = static_scene
    D, U = orc_tables
    Ct, dl = orc_colour
    h = lambda a: a.astype(np.float16).astype(np.float64)
    scene = orc.SceneTables(h(D), h(U), Ct.astype(np.float32), dl.astype(np.float32), scene32.cube,
                            scene32.cube_n, scene32.cube_dtype)
    t = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F16)
    try:
        disc = synth.WORKLOADS["static_256"]["disc"]
        og, gd, oo, od, mask = compare_render(orc, ctx, t, cube, scene, cam, disc,
                                              name=f"f16_{cam['width']}x{cam['height']}")
    finally:
        bh.bh_tables_free(t)
    check_stages(gd, od, mask)
    check_rgb(og, oo, od, mask, cam, "f16_tables")


def test_table_storage_precision_report(ctx, orc, orc_tables, orc_colour, static_scene):
    """Error of the linear-RGB image against the oracle reading FP64 tables, for
    the renderer reading FP32- and FP16-stored tables (the tables' own storage
    error, reported; FP32 must meet the parity tolerance)."""
    import json
    import os
    cube, scene32 = static_scene
    D, U = orc_tables
    Ct, dl = orc_colour
    wk = synth.WORKLOADS["static_256"]
    cam, disc = wk["camera"], wk["disc"]
    exact = orc.SceneTables(D, U, Ct.astype(np.float32), dl.astype(np.float32), scene32.cube,
                            scene32.cube_n, scene32.cube_dtype)
    oo, od, _ = orc.render(cam, disc, exact, exposure_stars=EXPOSURE_STARS, debug=True)
    mask = oracle_mask(od) | star_ill_conditioned(od, oo, cam)
    report = {}
    for name, storage in (("f32", bh.BH_F32), ("f16", bh.BH_F16)):
        t = bh.bh_precompute_tables(ctx, 512, 64, 32, storage)
        try:
            og, _ = gpu_render(ctx, t, cube, cam, disc)
        finally:
            bh.bh_tables_free(t)
        mean, mx, _ = image_error(og, oo, mask)
        report[name] = {"mean_rel": mean, "max_rel": mx}
    d = os.environ.get("BH_DUMP_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "table_storage_precision.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert report["f32"]["mean_rel"] <= RGB_MEAN_REL
    assert report["f16"]["mean_rel"] <= 0.05


def test_orbits_advance_matches_oracle(ctx, orc):
    """Device-resident free-fall orbits (Appendix C) follow the oracle's RK4."""
    import ctypes
    params = [(6.0, math.pi / 2, math.sqrt((1 / 6) / (2 * (5 / 6))), 0.3), (9.0, 1.3, 0.35, 0.6),
              (20.0, 2.2, 0.25, 1.0), (4.0, 2.8, 0.1, 0.0)]
    host = [bh.bh_orbit_init(r, d, v, chi, None, 1.0, 64, 48) for r, d, v, chi in params]
    buf = torch.frombuffer(bytearray(bh.orbits_to_bytes(host)), dtype=torch.uint8).cuda()
    bh.bh_orbits_advance(ctx, buf, len(host), 3.0, 60)
    bh.bh_orbits_advance(ctx, buf, len(host), 3.0, 60)
    torch.cuda.synchronize()
    got = (bh.Orbit * len(host)).from_buffer_copy(bytes(buf.cpu().numpy()))
    for (r, d, v, chi), g in zip(params, got):
        o = orc.orbit_init(r, d, v, chi)
        orc.orbit_advance(o, 3.0, 60)
        orc.orbit_advance(o, 3.0, 60)
        if o.r <= 1.05:
            continue
        assert g.r == pytest.approx(o.r, rel=1e-11)
        assert g.psi == pytest.approx(o.psi, rel=1e-11, abs=1e-12)
        assert g.t == pytest.approx(o.t, rel=1e-11)


def test_render_orbits_equals_batch(ctx, gpu_tables, static_scene):
    """Cameras computed on the device from orbits render as the same cameras
    staged from the host (FP64 set-up on both, rounded to FP32)."""
    cube, _ = static_scene
    host = [bh.bh_orbit_init(r, d, v, chi, None, 1.0, w, h)
            for (r, d, v, chi, w, h) in [(6.0, 1.5707963, 0.316, 0.3, 64, 48), (9.0, 1.3, 0.35, 0.6, 33, 17),
                                         (15.0, 2.0, 0.5, 1.2, 96, 64)]]
    buf = torch.frombuffer(bytearray(bh.orbits_to_bytes(host)), dtype=torch.uint8).cuda()
    disc = synth.disc()
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    outs = [torch.zeros((o.height, o.width, 4), device="cuda") for o in host]
    bh.bh_render_orbits(ctx, gpu_tables, cube, len(host), buf, disc, sh, outs)
    cams = [bh.camera_to_dict(bh.bh_orbit_camera(o)) for o in host]
    ref = [torch.zeros_like(o) for o in outs]
    bh.bh_render_batch(ctx, gpu_tables, cube, cams, disc, sh, ref)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6)


def test_served_orbits_equal_advance_then_render(gpu_tables, static_scene):
    """Viewers served on device-resident orbits: each request advances the
    viewer's orbit on the device and renders it; after three rounds the orbits
    and the frames equal bh_orbits_advance + bh_render_orbits on a copy."""
    cube, _ = static_scene
    c2 = bh.bh_create(0, 0)
    try:
        host = [bh.bh_orbit_init(r, d, v, chi, None, 1.0, w, h)
                for (r, d, v, chi, w, h) in [(6.0, 1.5707963, 0.316, 0.3, 64, 48), (9.0, 1.3, 0.35, 0.6, 33, 17),
                                             (15.0, 2.0, 0.5, 1.2, 96, 64), (7.0, 0.9, 0.2, -0.4, 40, 40)]]
        raw = bh.orbits_to_bytes(host)
        served = torch.frombuffer(bytearray(raw), dtype=torch.uint8).cuda()
        ref = served.clone()
        size = len(raw) // len(host)
        disc = synth.disc()
        sh = bh.make_shading(1.0, EXPOSURE_STARS)
        outs = [torch.zeros((o.height, o.width, 4), device="cuda") for o in host]
        refs = [torch.zeros_like(o) for o in outs]
        def submit_round():
            tickets = []
            for v, o in enumerate(host):
                for _ in range(100000):  # a viewer may hold one queued frame: retry until admitted
                    st, tk = bh.bh_serve_submit_orbit(c2, gpu_tables, cube, v, served.data_ptr() + v * size, 0.5,
                                                      4, o.width, o.height, disc, sh, outs[v])
                    if st == bh.BH_OK:
                        break
                    bh.bh_serve_flush(c2)
                assert st == bh.BH_OK
                tickets.append(tk)
            return tickets

        def reference_round():
            bh.bh_orbits_advance(c2, ref, len(host), 0.5, 4)
            bh.bh_render_orbits(c2, gpu_tables, cube, len(host), ref, disc, sh, refs)
            torch.cuda.synchronize()

        for rnd in range(2):  # one round at a time
            for tk in submit_round():
                assert bh.bh_serve_poll(c2, tk, 5_000_000)[0] == bh.BH_OK
            reference_round()
            for a, b in zip(outs, refs):
                assert torch.equal(a, b)
        # three rounds in flight at once on the three launch slots: each viewer's
        # orbit still advances in order, and its last frame is the third round's
        tickets = submit_round() + submit_round() + submit_round()
        for tk in tickets:
            assert bh.bh_serve_poll(c2, tk, 5_000_000)[0] == bh.BH_OK
        for _ in range(3):
            reference_round()
        torch.cuda.synchronize()
        for a, b in zip(outs, refs):
            assert torch.equal(a, b)
        assert torch.equal(served, ref)
        with pytest.raises(bh.BhError):
            bh.bh_serve_submit_orbit(c2, gpu_tables, cube, 0, served.data_ptr() + 1, 0.5, 4, 8, 8, disc, sh,
                                     outs[0])
    finally:
        bh.bh_destroy(c2)


def test_bounded_table_wait_reports_timeout(ctx, gpu_tables, static_scene):
    """Failure detection without a GPU fault: the injected table wait runs out,
    the kernel reports it through the status word, and the context renders
    normally afterwards."""
    cube, _ = static_scene
    cam = synth.camera(10.0, 80.0, width=64, height=64)
    sh = bh.make_shading(1.0, EXPOSURE_STARS)
    out = torch.zeros((64, 64, 4), device="cuda")
    assert bh.bh_check_status(ctx) == bh.BH_OK
    bh.bh_inject_fault(ctx, bh.BH_FAULT_TABLE_WAIT)
    bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, out)
    with pytest.raises(bh.BhError) as ei:
        bh.bh_check_status(ctx)
    assert ei.value.status == bh.BH_ERR_TIMEOUT
    ref = torch.zeros_like(out)
    bh.bh_render(ctx, gpu_tables, cube, cam, synth.disc(), sh, ref)
    assert bh.bh_check_status(ctx) == bh.BH_OK
    assert float(ref[..., 3].min()) == 1.0
