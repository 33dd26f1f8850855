"""Host-side pieces of bench.py, on the CPU: the grid option, the workload
name, and the ncu traffic lookup, which must refuse counters taken on another
grid or another kernel source, and whose committed counters belong to the
kernel source in the tree."""
import hashlib
import json
import os
from types import SimpleNamespace

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_grid_option_and_workload_name():
    assert bench.grid_of(SimpleNamespace(grid="")) == (600, 200, 120)
    assert bench.grid_of(SimpleNamespace(grid="300x200x120")) == (300, 200, 120)
    assert bench.workload_name((600, 200, 120)) == bench.WORKLOAD
    assert "300x200x120" in bench.workload_name((300, 200, 120))
    assert "600x200x120" not in bench.workload_name((300, 200, 120))


def test_traffic_counters_belong_to_the_kernel_source():
    """bench.py reports ncu traffic only from counters taken on the kernel
    source in the tree: with a matching hash they are used (on their own grid
    and tile only); after any kernel change they are refused (null)."""
    tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    src = open(os.path.join(ROOT, "paper_2311_05646_gb300", "csrc", "adg_kernels.cu"), "rb").read()
    tile = tr["tile"]
    current = tr["source_sha256"] == hashlib.sha256(src).hexdigest()
    for k in tr["kernels"]:
        v = bench._traffic(k, tile)
        if current:
            assert v is not None and v > 0
        else:
            assert v is None
        assert bench._traffic(k, tile, (300, 200, 120)) is None  # another grid
    assert bench._traffic("build", [64, 4, 4]) is None  # another tile


def test_small_grid_inputs_have_the_grating_shape():
    desc, ef, ea, w = bench.make_inputs((64, 40, 24))
    assert tuple(desc["grid"]["n"]) == (64, 40, 24)
    assert ef.shape == ea.shape == (3, 24, 40, 64)
    assert ef.dtype.name == "complex64" and len(w) == 3


def test_oracle_methods_on_a_small_grating():
    """The host baselines of the bench line: the analytic VJP on all cores and
    on one core, and the finite-difference method extrapolated to all the
    design's parameters -- which needs n + 1 eps builds and so is slower than
    the analytic one; the thread count is restored afterwards."""
    from oracle import oracle as O
    desc, ef, ea, w = bench.make_inputs((64, 40, 24))
    threads = O.num_threads()
    v, cores, sample, t = bench.oracle_sample(desc, ef, ea, w, target_s=0.2)
    assert v > 0 and cores == threads and t["fill_s"] > 0 and t["grad_s"] > 0
    m = bench.oracle_methods(desc, ef, ea, w, t, gpu_value=1e9, target_1core_s=0.2)
    assert O.num_threads() == threads
    assert m["params"] == len(desc["params"]) == 120
    for k in ("analytic_all_cores", "analytic_one_core", "fd_all_cores"):
        assert m[k]["value"] > 0, k
    assert m["analytic_one_core"]["cores"] == 1
    assert m["fd_all_cores"]["value"] < m["analytic_all_cores"]["value"] / 10
    assert abs(m["gpu_over_analytic"] * m["analytic_all_cores"]["value"] / 1e9 - 1) < 1e-9
    assert abs(m["gpu_over_fd"] * m["fd_all_cores"]["value"] / 1e9 - 1) < 1e-9
    assert m["analytic_over_fd"] > 10
