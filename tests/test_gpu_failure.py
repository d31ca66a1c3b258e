"""Failure detection without a GPU fault: a search whose stage barrier is
armed but never fed (test hook) must give up after its bounded wait, report
HD_ERR_TIMEOUT through the library status, and leave the context usable --
the next search on the same library is exact."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_16422_gb300 import build, hd as _hd
    build.build()
    return _hd


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("form,cluster,cta_group,tiles", [("popc", 0, 0, 1), ("tc_fp8", 1, 1, 1), ("tc_fp8", 2, 2, 1),
                                                          ("tc_fp4", 1, 1, 1), ("tc_fp4", 2, 2, 1),
                                                          ("tc_mxf4", 2, 2, 1), ("tc_mxf4", 2, 2, 2)])
def test_stalled_wait_times_out_then_recovers(hd, form, cluster, cta_group, tiles):
    rng = np.random.default_rng(12)
    D, W, n = 2048, 32, 3000
    refs = rng.integers(-2**63, 2**63, (n, W), dtype=np.int64)
    mz = rng.uniform(400, 600, n)
    z = np.full(n, 2, np.uint8)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library(ctx, dev(refs), dev(mz), dev(z))
    hd.hd_library_prepare(lib, form if form in ("tc_fp4", "tc_mxf4") else "tc_fp8")
    hd.hd_library_set_schedule(lib, 0, 0, cluster, cta_group)
    hd.hd_library_set_stage_tiles(lib, tiles)
    q, qm, qz = dev(refs[:300]), dev(mz[:300]), dev(z[:300])
    hd.hd_library_set_wait_limit(lib, 0.05)
    hd.hd_library_inject_stall(lib, 1)
    hd.hd_search_open(lib, q, qm, qz, 50.0, "da", 3, form=form)
    torch.cuda.synchronize()          # the kernel returned: no hang
    with pytest.raises(hd.HDError) as e:
        lib.status()
    assert e.value.status == hd.HD_ERR_TIMEOUT
    lib.status()                      # cleared
    i, d = hd.hd_search_open(lib, q, qm, qz, 50.0, "da", 3, form=form)
    torch.cuda.synchronize()
    lib.status()
    oi, od = oracle.search(D, refs.view(np.uint64), mz, z, refs[:300].view(np.uint64), mz[:300], z[:300], 50.0,
                           "da", 3)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(hd.as_u16(d), od)


@pytest.mark.parametrize("form", ["tc_fp4", "popc"])
def test_stalled_dot_search_times_out_then_recovers(hd, form):
    """The same bounded-wait path for the multi-bit dot-product search (the
    tensor-core form and the popcount form on bit planes)."""
    rng = np.random.default_rng(13)
    D, n, bits = 1024, 3000, 3
    R = rng.integers(-3, 4, (n, D)).astype(np.int8)
    mz = rng.uniform(400, 600, n)
    z = np.full(n, 2, np.uint8)
    ctx = hd.Ctx(D, 4, 10, D // 2, 0)
    lib = hd.hd_build_library_multibit(ctx, dev(R), dev(mz), dev(z), bits)
    hd.hd_library_prepare(lib, form)
    q, qm, qz = dev(R[:300]), dev(mz[:300]), dev(z[:300])
    hd.hd_library_set_wait_limit(lib, 0.05)
    hd.hd_library_inject_stall(lib, 1)
    hd.hd_search_dot(lib, q, qm, qz, 50.0, "da", 3, form)
    torch.cuda.synchronize()
    with pytest.raises(hd.HDError) as e:
        lib.status()
    assert e.value.status == hd.HD_ERR_TIMEOUT
    lib.status()
    i, sc = hd.hd_search_dot(lib, q, qm, qz, 50.0, "da", 3, form)
    torch.cuda.synchronize()
    lib.status()
    oi, osc = oracle.search_dot(R, mz, z, R[:300], mz[:300], z[:300], 50.0, "da", 3)
    assert np.array_equal(hd.as_u32(i), oi) and np.array_equal(sc.cpu().numpy(), osc)
