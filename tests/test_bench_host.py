"""bench.py host logic: the per-kernel source hash that keys the committed ncu
traffic figures (checked on a scratch copy of the kernel sources), and the
reference arm's JSON line (the oracle on the host cores, no GPU)."""

import os
import shutil

import bench


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2402_09481_gb300", "csrc")
    dst = tmp_path / "paper_2402_09481_gb300" / "csrc"
    shutil.copytree(src, dst)
    (tmp_path / "profiles").mkdir()
    return dst


KERNELS = ("k_pass", "k_middle_f30", "k_vn_write", "k_rsh", "k_ss_gf2", "k_middle_f25", "k_pass_fwd_bits_f25",
           "k_pack_tail", "k_cluster_f25", "k_batch")


def _hashes():
    return {k: bench.kernel_source_hash(k) for k in KERNELS}


def test_hash_follows_own_unit(tmp_path, monkeypatch):
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = _hashes()
    assert before["k_pass"] == before["k_middle_f30"]          # one family
    assert before["k_middle_f25"] == before["k_pass_fwd_bits_f25"]
    assert len({before[k] for k in ("k_pass", "k_vn_write", "k_rsh", "k_ss_gf2", "k_middle_f25", "k_pack_tail",
                                    "k_cluster_f25", "k_batch")}) == 8

    with open(csrc / "cm_trevisan.cu", "a") as f:
        f.write("\nstatic const int edit_marker = 1;\n")
    after = _hashes()
    assert after["k_rsh"] != before["k_rsh"]
    assert all(after[k] == before[k] for k in ("k_pass", "k_vn_write", "k_ss_gf2"))

    with open(csrc / "cm_api.cu", "a") as f:                  # the planner
        f.write("\nstatic const int edit_marker = 1;\n")
    after2 = _hashes()
    assert all(after2[k] != after[k] for k in ("k_pass", "k_middle_f25", "k_pack_tail", "k_cluster_f25", "k_batch"))
    assert all(after2[k] == after[k] for k in ("k_rsh", "k_vn_write", "k_ss_gf2"))

    with open(csrc / "cm_pass25.cu", "a") as f:               # the 5 * 2^25 + 1 column passes and middle
        f.write("\nstatic const int edit_marker = 1;\n")
    after25 = _hashes()
    assert after25["k_middle_f25"] != after2["k_middle_f25"] and after25["k_pass_fwd_bits_f25"] != after2[
        "k_pass_fwd_bits_f25"]
    assert all(after25[k] == after2[k] for k in ("k_pack_tail", "k_cluster_f25", "k_batch", "k_rsh", "k_vn_write"))
    with open(csrc / "cm_batch.cu", "a") as f:                # the work list
        f.write("\nstatic const int edit_marker = 1;\n")
    afterb = _hashes()
    assert afterb["k_batch"] != after25["k_batch"] and afterb["k_pass"] != after25["k_pass"]
    assert all(afterb[k] == after25[k] for k in ("k_middle_f25", "k_pack_tail", "k_cluster_f25", "k_ss_gf2"))
    after2 = afterb

    with open(csrc / "cm_internal.h", "a") as f:              # a header every unit includes
        f.write("\nstatic const int edit_marker = 1;\n")
    after3 = _hashes()
    assert all(after3[k] != after2[k] for k in after3)

    (csrc / "unused_new.cuh").write_text("// included by nothing\n")   # no kernel's source
    assert _hashes() == after3

    with open(csrc / "cm_internal.h", "a") as f:              # comments and blank lines only
        f.write("\n// a comment\n/* and a\n   block comment */\n\n")
    assert _hashes() == after3


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h_rsh, h_vn = bench.kernel_source_hash("k_rsh"), bench.kernel_source_hash("k_vn_write")
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        "# kernel workload bytes hash\n"
        f"k_rsh trevisan 1234 {h_rsh}\n"
        f"k_vn_write von_neumann 5678 {h_vn}\n")
    assert bench.ncu_traffic("k_rsh", "trevisan") == 1234.0
    assert bench.ncu_traffic("k_vn_write", "von_neumann") == 5678.0
    assert bench.ncu_traffic("k_rsh", "von_neumann") is None
    with open(csrc / "cm_vn.cu", "a") as f:
        f.write("\nstatic const int edit_marker = 1;\n")
    assert bench.ncu_traffic("k_vn_write", "von_neumann") is None
    assert bench.ncu_traffic("k_rsh", "trevisan") == 1234.0


def test_reference_arm_json_line():
    # the reference arm times the oracle on the host cores (no GPU): one JSON
    # line with the contract's keys, the ratio's inputs and no host copies
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    for k in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
