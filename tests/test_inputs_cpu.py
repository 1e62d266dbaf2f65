"""The synthetic inputs are the recipe the design notes state: seeded,
reproducible, closed, and of the documented sizes (the benchmark's workload,
its oracle-sized case and the large parity configurations)."""
import numpy as np

from synth import meshes as M


def _closed(m):
    return M.watertight_edges(m.tris) and np.isfinite(m.verts).all()


def test_benchmark_workload_recipe():
    import bench
    w = bench.workload("sdf2m-1024", 0)
    assert (w["N"], w["depth"], w["sweeps"], w["mesh"].n_tris) == (1024, 14, 3, 2029088)
    assert _closed(w["mesh"])
    assert "2,029,088 triangles" in w["name"] and "1024^3" in w["name"]
    m = bench.workload("sdf200k-512", 0)
    assert (m["N"], m["depth"], m["mesh"].n_tris) == (512, 10, 202244) and _closed(m["mesh"])
    again = bench.workload("sdf200k-512", 0)["mesh"]
    assert np.array_equal(again.verts, m["mesh"].verts) and np.array_equal(again.tris, m["mesh"].tris)
    other = bench.workload("sdf200k-512", 1)["mesh"]     # each rank meshes its own seed
    assert other.n_tris != m["mesh"].n_tris or not np.array_equal(other.verts, m["mesh"].verts)
    s = bench.workload("torus4k-64", 0)
    assert (s["N"], s["depth"], s["mesh"].n_tris) == (64, 4, 4096) and _closed(s["mesh"])


def test_large_configuration_sizes():
    m1 = M.sdf_union_1m()
    assert m1.n_tris == 1059784 and _closed(m1)
    m2 = M.sdf_union_2m()
    assert m2.n_tris == 2029088 and _closed(m2)
