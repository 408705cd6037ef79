"""The benchmark's work and byte accounting (CPU): the counts behind its roofline figures,
checked against hand-computed values for the pml-160 workload (160 x 160 x 128, one
interface per axis at node 79, so blocks of 79 and 80 nodes, 4 RHS)."""
import json
import os

from paper_1909_01299_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bulk_transform_multiply_adds():
    import bench
    w = W.pml_160x160x128()
    # per launch: RHS x planes x rows outside the other axis' interface x sum of n^2 over blocks
    per_launch = 4 * 128 * 159 * (79 * 79 + 80 * 80)
    assert bench.bulk_macs(w, 4) == [per_launch] * 4


def test_tensor_core_bytes_per_launch():
    import bench
    w = W.pml_160x160x128()
    values = 159 * 159 * 128 * 4
    # one solve: 24 + 16 + 16 + 24 B per value over 4 launches
    assert bench.tc_bytes_per_launch(w, 4, 0) == values * 80 / 4
    # with one accumulating correction: + 24 + 16 + 16 + 40 B over 4 more launches
    assert bench.tc_bytes_per_launch(w, 4, 1) == values * (80 + 96) / 8


def test_tf32_peak_follows_the_measured_bf16_figure():
    import bench
    peak, src = bench.tf32_peak()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        assert src.startswith("measured")
    else:                                   # the peaks file is written per machine
        bf16 = 1900.0
        assert src.startswith("fallback")
    assert abs(peak - bf16 * 1.1 / 2.25) < 1e-9


def test_traffic_records_are_dropped_for_changed_sources(tmp_path, monkeypatch):
    import bench
    w_name = "pml-160x160x128-2x2blocks-4rhs-fp64"
    rec = {"xform_tc_kernel": {"source_sha": "0" * 16, "workload": w_name, "bytes_per_launch": 1}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    src = tmp_path / "paper_1909_01299_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "hz_xform_tc.cu").write_text("// another source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("xform_tc_kernel", w_name, "hz_xform_tc.cu") is None
    rec["xform_tc_kernel"]["source_sha"] = bench.kernel_source_hash("hz_xform_tc.cu")
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.profiled_traffic("xform_tc_kernel", w_name, "hz_xform_tc.cu") == 1


def test_benchmark_workload_counts():
    # 320 x 320 x 200, interfaces at 79, 159, 239: blocks of 79, 79, 79 and 80 nodes, 8 RHS;
    # every block is uniform with n + 1 = 80 or 81, so all take the fast sine transform
    import math
    import bench
    w = bench.bench_workload()
    assert (w.nx, w.ny, w.nz, w.nrhs) == (320, 320, 200, 8)
    per_launch = 8 * 200 * 317 * (3 * 79 * 79 + 80 * 80)
    assert bench.bulk_macs(w, 8) == [per_launch] * 4
    assert bench.real_tables(w)
    assert bench.uniform_blocks(w.hx, w.x_iface) == [True] * 4
    assert [bench.fast_sine_ok(n) for n in (79, 80, 12, 127, 128)] == [True, True, False, True, False]
    rows = 8 * 200 * 317
    fft = lambda N: 5 * N * math.log2(N) + 9 * (N - 1)
    dense, fast, all_fast = bench.fp64_transform_work(w, 8)
    assert all_fast and dense == 0
    assert abs(fast - rows * (3 * fft(80) + fft(81))) < 1e-6 * fast
    st = {k: (0.0, 0) for k in ("fwd", "pass_a", "edges", "iface_residual", "global", "pass_b", "inv",
                                "iface_out", "residual")}
    st["fwd"] = (2.0, 2)
    st["inv"] = (2.0, 2)
    roof = bench.fp64_roofline(w, 8, st)
    assert roof["kernel"].startswith("dst_kernel")
    assert abs(roof["achieved"] - fast / 1e-3 / 1e12) < 1e-9
    one = bench.one_rhs(w, 3)
    assert one.nrhs == 1 and (one.f[0] == w.f[3]).all()


def test_pml_workload_uses_the_dense_count():
    # the PML rim makes every block non-uniform (complex tables): 8 n flops per value
    import bench
    w = W.pml_160x160x128()
    dense, fast, all_fast = bench.fp64_transform_work(w, 4)
    assert fast == 0 and not all_fast
    assert dense == 4 * 128 * 159 * (79 * 79 + 80 * 80) * 8


def test_tensor_core_mma_work_and_kernel_names():
    # the MMA flops of a step's transforms: interleaved complex GEMM 8 flops per complex
    # multiply-add, the real-table kernel 4 (its two real products of K = N = n); 3 TF32 products
    import bench
    w = bench.bench_workload()
    per = 8 * 200
    sq = 3 * 79 * 79 + 80 * 80
    inter = 3 * per * (2 * 317 * sq * 8 + 2 * 317 * sq * 8)
    assert bench.tc_mma_flops(w, 8, False) == inter
    assert bench.tc_mma_flops(w, 8, True) == inter // 2
    assert bench.real_block_flags(w.hx, w.x_iface) == [True] * 4
    st = {k: (0.0, 0) for k in ("fwd", "pass_a", "edges", "iface_residual", "global", "pass_b", "inv",
                                "iface_out", "residual")}
    st["fwd"] = (1.0, 2)
    st["inv"] = (1.0, 2)
    assert bench.tc_roofline(w, 8, st, 0, True)["kernel"].startswith("xform_tcr_kernel")
    assert bench.tc_roofline(w, 8, st, 0, False)["kernel"].startswith("xform_tc_kernel ")
    # pml-160: the blocks reach into the complex rim steps, so no table is real
    p = W.pml_160x160x128()
    assert bench.real_block_flags(p.hx, p.x_iface) == [False, False]
    assert bench.tc_mma_flops(p, 4, True) == bench.tc_mma_flops(p, 4, False)
    assert bench.tc_roofline(p, 4, st, 1, True)["kernel"].startswith("xform_tc_kernel ")
