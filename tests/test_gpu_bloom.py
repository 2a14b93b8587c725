"""The CUDA bloom (Sec. 3.4.3 lens glare, bh_bloom) against the FP64 oracle
(oracle/bloom.py) on the same FP32 input frames, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import bloom as ob
from paper_2010_08735_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2010_08735_gb300 import bh  # noqa: E402

BLOOM_REL = 1e-5  # FP32 arithmetic over a few dozen operations per pixel


@pytest.fixture(scope="module")
def ctx():
    c = bh.bh_create(0, 0)
    yield c
    bh.bh_destroy(c)


def hdr_frame(H, W, seed):
    """Sky-like test frame: a dim smooth background, a few very bright points
    (stars, 1e4 x brighter) and a bright band (a disc)."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W, 4), dtype=np.float32)
    yy, xx = np.mgrid[0:H, 0:W]
    img[..., 0] = 1e-3 * (1 + np.sin(xx / 7.0))
    img[..., 1] = 1e-3 * (1 + np.cos(yy / 5.0))
    img[..., 2] = 2e-3
    band = np.abs(yy - 0.6 * H) < 0.05 * H + 1
    img[band, :3] += np.array([0.8, 0.5, 0.2], dtype=np.float32)
    for _ in range(max(3, H * W // 2000)):
        y, x = rng.integers(0, H), rng.integers(0, W)
        img[y, x, :3] += rng.uniform(1, 10, 3).astype(np.float32) * 10.0
    img[..., 3] = 1.0
    return img


def compare(gpu, ref):
    floor = 1e-6 * np.abs(ref).max()
    rel = np.abs(gpu[..., :3].astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)
    return float(rel.max())


def test_weights_match_oracle():
    for fov, H, K in [(math.radians(60), 1080, 6), (math.radians(60), 2160, 8), (0.3, 97, 3), (1.0, 1, 0)]:
        assert np.allclose(bh.bh_bloom_weights(fov, H, K), ob.bloom_weights(fov, H, K), rtol=1e-12, atol=1e-15)


# (300, 520, 10): the maximum level count (levels 8..10 one grid-wide pass
# each, the composite's staged rows at their largest); (129, 257, 8): odd
# sizes at every level past the region depth
@pytest.mark.parametrize("H,W,K", [(256, 256, 6), (61, 97, 4), (1, 1, 2), (33, 17, 0), (1080, 1920, 6),
                                   (300, 520, 10), (129, 257, 8)])
def test_bloom_matches_oracle(ctx, H, W, K):
    img = hdr_frame(H, W, seed=H * 7 + W)
    w = bh.bh_bloom_weights(math.radians(60), max(H, 2), K)
    inp = torch.from_numpy(img).cuda()
    out = torch.empty_like(inp)
    bh.bh_bloom(ctx, inp, out, W, H, w)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = ob.bloom(img, w)
    assert compare(got, ref) <= BLOOM_REL
    assert np.all(got[..., 3] == 1.0)
    if K == 0:
        assert np.array_equal(got[..., :3], img[..., :3])


def test_bloom_in_place_and_rendered_frame(ctx):
    """In place on a rendered frame (the 256^2 static view), twice in a row
    with another size between (the context's pyramid scratch is reused)."""
    wk = synth.WORKLOADS["static_256"]
    cam = wk["camera"]
    t = bh.bh_precompute_tables(ctx, 512, 64, 32, bh.BH_F32)
    cube = bh.bh_build_star_cubemap(ctx, synth.stars(wk["n_stars"], wk["star_seed"]), wk["cube_n"], bh.BH_F16)
    try:
        frame = torch.zeros((256, 256, 4), device="cuda")
        bh.bh_render(ctx, t, cube, cam, wk["disc"], bh.make_shading(1.0, 0.05), frame)
        torch.cuda.synchronize()
        img = frame.cpu().numpy()
        w = bh.bh_bloom_weights(cam["fov_y"], 256, 5)
        ref = ob.bloom(img, w)
        for _ in range(2):
            buf = torch.from_numpy(img).cuda()
            bh.bh_bloom(ctx, buf, buf, 256, 256, w)
            torch.cuda.synchronize()
            assert compare(buf.cpu().numpy(), ref) <= BLOOM_REL
            other = torch.from_numpy(hdr_frame(40, 70, 1)).cuda()
            bh.bh_bloom(ctx, other, other, 70, 40, bh.bh_bloom_weights(cam["fov_y"], 40, 3))
    finally:
        bh.bh_cubemap_free(cube)
        bh.bh_tables_free(t)


def test_bloom_rejects_bad_arguments(ctx):
    buf = torch.zeros((8, 8, 4), device="cuda")
    with pytest.raises(bh.BhError):
        bh.bh_bloom(ctx, buf, buf, 8, 8, np.ones(12))  # 11 levels > 10
    with pytest.raises(bh.BhError):
        bh.bh_bloom(ctx, buf, buf, 0, 8, np.ones(2))
    with pytest.raises(bh.BhError):
        bh.bh_bloom_weights(0.0, 8, 2)


def test_bloom_barrier_timeout_is_reported_and_context_recovers(ctx):
    """Failure detection without a GPU fault: one block of the next bloom never
    arrives at its first grid barrier (bh_inject_fault); every block's bounded
    wait (2 ms) runs out, the blocks stop, bh_check_status reports
    BH_ERR_TIMEOUT, and the next bloom on the context is correct."""
    H, W = 120, 200
    img = hdr_frame(H, W, 5)
    w = bh.bh_bloom_weights(math.radians(60), H, 3)
    inp = torch.from_numpy(img).cuda()
    out = torch.zeros_like(inp)
    bh.bh_inject_fault(ctx, bh.BH_FAULT_BLOOM_BARRIER)
    bh.bh_bloom(ctx, inp, out, W, H, w)
    torch.cuda.synchronize()
    with pytest.raises(bh.BhError) as ei:
        bh.bh_check_status(ctx)
    assert ei.value.status == bh.BH_ERR_TIMEOUT
    bh.bh_bloom(ctx, inp, out, W, H, w)
    torch.cuda.synchronize()
    assert bh.bh_check_status(ctx) == bh.BH_OK
    assert compare(out.cpu().numpy(), ob.bloom(img, w)) <= BLOOM_REL
