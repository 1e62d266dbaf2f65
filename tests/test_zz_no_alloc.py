"""The outer-volume entry point that allocates no device memory.

It serves callers that cannot allocate device memory once running (a real-time
collision loop on a fixed memory budget, or a framework that owns the whole
device pool).  Its counts must equal those of the regular entry point, call
after call, even though every call reuses the same fixed scratch array.
This file is collected last so that a failure here leaves every other test
already run; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from synth import meshes as M
from tests import pins

pytestmark = pytest.mark.gpu


def _boxes(rng, K, lo, hi, half_lo, half_hi):
    out = np.zeros((K, 12), dtype=np.float32)
    for i in range(K):
        R = pins.random_rotation(rng)
        out[i, :3] = rng.uniform(lo, hi)
        out[i, 3:6] = R[0]
        out[i, 6:9] = R[1]
        out[i, 9:12] = rng.uniform(half_lo, half_hi, 3)
    return out


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2203_10521_gb300 as P
    ctx = P.Context(0)
    m = M.torus_4096()
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 64)
    rng = np.random.Generator(np.random.PCG64(99))
    # two different batches in a row: the second call must not see the first's scratch
    batches = [_boxes(rng, 700, [-1.6, -1.6, -0.6], [1.6, 1.6, 0.6], 0.0, 0.5),
               _boxes(rng, 123, [-1.0, -1.0, -0.3], [1.0, 1.0, 0.3], 0.05, 1.2)]
    free_before = None
    for i, boxes in enumerate(batches + batches[:1]):
        q = ctx.quantize_boxes(lat, boxes)
        dq = torch.from_numpy(q.view(np.uint8).copy()).cuda()
        ref_c, ref_p = ctx.outer_volume_q(lat, dq, want_points=True)   # regular path (device arrays)
        torch.cuda.synchronize()
        if i == 1:
            free_before = torch.cuda.mem_get_info()[0]
        cnt = torch.full((len(boxes),), -1, dtype=torch.int64, device="cuda")
        pts = torch.full((len(boxes),), -1, dtype=torch.int64, device="cuda")
        ctx.outer_volume_q_noalloc(lat, dq, cnt, pts)
        ctx.synchronize()
        assert torch.equal(cnt, ref_c), f"call {i}: counts differ"
        assert torch.equal(pts, ref_p), f"call {i}: point counts differ"
    # no device memory was taken by the no-allocation calls after set-up
    ctx.outer_volume_q_noalloc(lat, dq, cnt, None)
    ctx.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    # batches above the fixed maximum are refused with a clear error
    big = torch.zeros(4097 * 88, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4097, dtype=torch.int64, device="cuda")
    with pytest.raises(P.ObbError) as e:
        ctx.outer_volume_q_noalloc(lat, big, out)
    assert e.value.code == -3 and "4096" in str(e.value)
    # the largest batch allowed fills every scratch region
    q = ctx.quantize_boxes(lat, _boxes(rng, 4096, [-1.6, -1.6, -0.6], [1.6, 1.6, 0.6], 0.0, 0.8))
    dq = torch.from_numpy(q.view(np.uint8).copy()).cuda()
    ref_c, ref_p = ctx.outer_volume_q(lat, dq, want_points=True)
    cnt = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
    pts = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
    ctx.outer_volume_q_noalloc(lat, dq, cnt, pts)
    ctx.synchronize()
    assert torch.equal(cnt, ref_c) and torch.equal(pts, ref_p)
    # arrays the entry point cannot use are refused before any launch
    with pytest.raises(ValueError):
        ctx.outer_volume_q_noalloc(lat, dq.cpu(), cnt)
    with pytest.raises(ValueError):
        ctx.outer_volume_q_noalloc(lat, dq, cnt[:100])
    with pytest.raises(ValueError):
        ctx.outer_volume_q_noalloc(lat, dq[:-1], cnt)
    lat.free()
    # the per-box row axis reads the lattice's y- and z-row copies through the same scratch
    try:
        ctx.set_counting_axis(-1)
        lat = ctx.build_occupancy(mesh, 64)
        dq = torch.from_numpy(ctx.quantize_boxes(lat, batches[0]).view(np.uint8).copy()).cuda()
        ref_c = ctx.outer_volume_q(lat, dq)
        cnt = torch.full((len(batches[0]),), -1, dtype=torch.int64, device="cuda")
        ctx.outer_volume_q_noalloc(lat, dq, cnt)
        ctx.synchronize()
        assert torch.equal(cnt, ref_c)
    finally:
        ctx.set_counting_axis(0)
    lat.free()
    mesh.free()
    ctx.close()
