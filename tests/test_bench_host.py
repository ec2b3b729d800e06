"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes of the dominant kernel's
roofline line and the rule that a committed DRAM-traffic record is reported only while the
kernel source it was captured from is unchanged."""
import hashlib
import os

import bench
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_angular_step_roofline_bytes_config2():
    cfg = W.CONFIGS["c2"]
    g = cfg["grid"]
    npts = g["NR"] * g["nr"] * g["ngamma"]
    nblk = sum(min(J, cfg["omega_max"]) + 1 for J in cfg["J"]) * cfg["nelec"]
    assert nblk == 11
    bound, b = bench.kernel_roofline("angular_tc", 4, npts, nblk, g["ngamma"], 1,
                                     cfg["analysis"]["nE"], 128, 0)
    assert bound == "hbm"
    # read q_k and q_(k-1), write q_(k+1), FP32, for every grid value of every block, plus
    # the potential V[gamma][r][R] of the J once
    assert b == 3 * 4 * npts * nblk + 4 * npts
    assert abs(b / 1e9 - 0.6418) < 1e-4


def test_traffic_record_follows_its_kernel_source():
    rec = os.path.join(ROOT, "profiles", "traffic_angular_tc_c2_mixed.txt")
    fields = {}
    for ln in open(rec):
        if ln.strip() and not ln.startswith("#"):
            k, _, v = ln.strip().partition(" ")
            fields[k] = v.strip()
    with open(os.path.join(ROOT, fields["source"]), "rb") as f:
        same = hashlib.sha1(f.read()).hexdigest() == fields["source_sha1"]
    t = bench.captured_traffic("angular_tc")
    if same:
        assert t == float(fields["dram_bytes"])
        # DRAM bytes of a launch lie between the method minimum and the design bytes with t
        assert 0.6418e9 < t < 0.8495e9
    else:
        assert t is None
