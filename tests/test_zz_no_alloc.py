"""The allocation-free cube-map build, called through the C ABI, against the
allocating entry point (bh_build_star_cubemap) on the same stars.

This entry point is for callers that cannot allocate device memory
themselves (their application owns all device memory through its own pool,
or they run on threads that must not call cudaMalloc).  Its scratch is one
static device array shared by every call, so two calls in a row are checked:
the second must not see the first call's accumulators.  Collected last (file
name), so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2010_08735_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2010_08735_gb300 import bh  # noqa: E402


def reference_records(ctx, stars, N, dtype):
    c = bh.bh_build_star_cubemap(ctx, stars, N, dtype)
    try:
        return bh.bh_cubemap_copy_out(c, N)
    finally:
        bh.bh_cubemap_free(c)


def test_noalloc_cubemap_matches_allocating_build_twice():
    """Calls in a row on the one static scratch array, each against the
    allocating build: a full-size face, then the same face size with fewer
    stars (the accumulators must have been cleared, not summed onto), another
    storage type, an empty star list at face size 1 (no mip levels, NULL star
    pointer) and a few stars at face size 1."""
    ctx = bh.bh_create(0, 0)
    try:
        calls = [(synth.stars(20000, seed=21), 128, bh.BH_F16),
                 (synth.stars(3000, seed=23), 128, bh.BH_F16),
                 (synth.stars(3000, seed=22), 64, bh.BH_BF16),
                 (np.zeros((0, 5), dtype=np.float32), 1, bh.BH_F16),
                 (synth.stars(5, seed=24), 1, bh.BH_BF16)]
        for stars, N, dtype in calls:
            dst = torch.from_numpy(stars).cuda()
            rec = torch.empty((bh.bh_cubemap_records(N), 4), dtype=torch.int16, device="cuda")
            bh.bh_build_star_cubemap_noalloc(dst, N, dtype, rec)
            torch.cuda.synchronize()
            got = rec.cpu().numpy().view(np.uint16)
            ref = reference_records(ctx, stars, N, dtype)
            # the cube map is integer/bit work: the tolerance is exact equality
            assert np.array_equal(got, ref), (len(stars), N, dtype)
    finally:
        bh.bh_destroy(ctx)


def test_noalloc_rejects_faces_beyond_its_scratch():
    dst = torch.from_numpy(synth.stars(10, seed=1)).cuda()
    rec = torch.empty((bh.bh_cubemap_records(256), 4), dtype=torch.int16, device="cuda")
    with pytest.raises(bh.BhError) as ei:
        bh.bh_build_star_cubemap_noalloc(dst, 256, bh.BH_F16, rec)
    assert ei.value.status == bh.BH_ERR_INVALID_ARG
    assert "128" in str(ei.value)
