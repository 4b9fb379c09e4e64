"""The bench's roofline accounting (CPU only): algorithmic bytes per node of each stage
kernel, written out from the arrays each kernel consumes and produces (3D, N = 5: one
face point per node; nv = 6 conserved variables, nl = 5 lifted ones), and the rule that
an ncu summary counts only for the kernel sources it was taken on."""
import os

import pytest

import bench


def test_box_fp32_bulk_bytes():
    kb = bench.kernel_bytes_per_node(3, 5, 4)
    # k_lift1: float shadow (nv + 1) in, c traces in, T and dc/dn traces out
    assert kb["k_lift1"] == 4 * 7 + 4 * 1 + 4 * 2
    # k_lift2vol: shadow, pass-1 traces (nl), pass-2 traces (2), U_t volume part (nv) out,
    # face data (2 nv + 1) out
    assert kb["k_lift2vol"] == 4 * 7 + 4 * 5 + 4 * 2 + 4 * 6 + 4 * 13
    # k_surf_rk: face data in, U_t volume part in, U and G in and out in FP64, new pass-1
    # traces and the float shadow out
    assert kb["k_surf_rk"] == 4 * 13 + 4 * 6 + 8 * 6 * 4 + 4 * 5 + 4 * 7
    assert sum(kb.values()) == 488


def test_box_fp64_bytes():
    kb = bench.kernel_bytes_per_node(3, 5, 8)
    assert kb["k_lift1"] == 8 * 6 + 8 * 1 + 8 * 2
    assert kb["k_lift2vol"] == 8 * 6 + 8 * 5 + 8 * 2 + 8 * 6 + 8 * 13
    assert kb["k_surf_rk"] == 8 * 13 + 8 * 6 + 8 * 6 * 4 + 8 * 5


def test_hllc_and_curved_bytes():
    box, hllc = bench.kernel_bytes_per_node(3, 5, 4), bench.kernel_bytes_per_node(3, 5, 4, "hllc")
    # two more face-data values per face point (convective pressure, sound speed)
    assert hllc["k_lift2vol"] - box["k_lift2vol"] == 8
    assert hllc["k_surf_rk"] - box["k_surf_rk"] == 8
    cv = bench.kernel_bytes_per_node(3, 5, 4, curved=True)
    geo = 4 * (9 + 1) + 4 * 3  # J a^i and 1/J per node, J a^dir per face point
    assert cv == {"k_lift1c": box["k_lift1"] + geo, "k_lift2volc": box["k_lift2vol"] + geo,
                  "k_surf_rk": box["k_surf_rk"] + 4}
    cvh = bench.kernel_bytes_per_node(3, 5, 4, "hllc", curved=True)
    assert cvh["k_surf_rk"] == hllc["k_surf_rk"] + 4 + 4 * 3  # 1/J and the unit normal's face metric


def test_two_dimensional_face_points_per_node():
    # 2D, N = 3: 2 d / (N + 1) = 1 face point per node as well; N = 4: 0.8
    kb3, kb4 = bench.kernel_bytes_per_node(2, 3, 4), bench.kernel_bytes_per_node(2, 4, 4)
    assert kb3["k_lift1"] == 4 * 6 + 4 * 1 + 4 * 2
    assert kb4["k_lift1"] == pytest.approx(4 * 6 + 0.8 * (4 + 8))


def test_ncu_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "profiles")
    csrc = tmp_path / "paper_2208_05310_gb300" / "csrc"
    os.makedirs(csrc)
    for fn in ("dgk_common.cuh", "dgk_kernels.cuh", "dgk_curved.cuh"):
        (csrc / fn).write_text("// " + fn + "\n")
    sha = bench.kernel_sources_sha()
    body = f"kernel_source_sha1: {sha}\ndram_bytes_per_launch_full: 123456\n"
    (tmp_path / "profiles" / "k_lift2vol_c5_fp32.txt").write_text(body)
    assert bench.ncu_traffic("k_lift2vol", "c5_fp32") == pytest.approx(123456)
    (csrc / "dgk_kernels.cuh").write_text("// changed\n")
    assert bench.ncu_traffic("k_lift2vol", "c5_fp32") is None
    assert bench.ncu_traffic("k_surf_rk", "c5_fp32") is None


def test_batch_traffic_follows_the_batched_sources(tmp_path, monkeypatch):
    """The batched form's DRAM bytes per stage count only while the stage kernels and the
    batched kernels are the sources the summary was taken on."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "profiles")
    csrc = tmp_path / "paper_2208_05310_gb300" / "csrc"
    os.makedirs(csrc)
    for fn in ("dgk_common.cuh", "dgk_kernels.cuh", "dgk_batch.cu"):
        (csrc / fn).write_text("// " + fn + "\n")
    body = f"kernel_source_sha1: {bench.kernel_sources_sha(batch=True)}\ndram_bytes_per_stage: 777\n"
    (tmp_path / "profiles" / "k_batch_phase_c4_fp32.txt").write_text(body)
    assert bench.batch_traffic("c4") == pytest.approx(777)
    assert bench.batch_traffic("c4s") is None  # no summary of that workload
    (csrc / "dgk_batch.cu").write_text("// changed\n")
    assert bench.batch_traffic("c4") is None


def test_l2_note_says_when_a_workload_fits_in_l2():
    assert bench.l2_note(1.36e9).startswith("inputs larger than L2")
    assert "fit in L2" in bench.l2_note(4.1e6)
