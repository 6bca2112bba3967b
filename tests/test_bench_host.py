"""Host logic of the benchmark (no GPU): the ncu records are used only for
the kernel source they were taken on, launch labels, the ALU roofline and
streaming-view arithmetic and the extras selection."""

import hashlib
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _source_sha():
    src = b"".join(open(os.path.join(ROOT, "paper_2305_04180_gb300", "csrc", f), "rb").read()
                   for f in ("sg_device.cuh", "sg_sim.cu"))
    return hashlib.sha1(src).hexdigest()[:16]


def _records():
    out = []
    for line in open(os.path.join(ROOT, "profiles", "roofline_traffic.txt")):
        line = line.strip()
        if line.startswith("kernel="):
            out.append(dict(tok.split("=", 1) for tok in line.split(" ") if "=" in tok))
    return out


def test_traffic_records_are_used_only_on_their_kernel_source():
    """A record taken on the current kernel source gives its read + write
    bytes for exactly its workload and launch (at least the 153 B per
    env-step of materialised outputs); a record of another source is never
    used (the benchmark then reports no traffic)."""
    recs = _records()
    assert recs
    sha = _source_sha()
    for r in recs:
        n, K = int(r["n_envs"]), int(r["steps_per_launch"])
        got = bench._recorded(n, K, r["kernel"], r["launch"])
        if r["source_sha1"] == sha:
            traffic = int(r["dram_bytes_read"]) + int(r["dram_bytes_write"])
            assert got["dram_bytes"] == traffic and got["scale"] == 1.0
            if r["kernel"] != "k_step":  # the rollout writes its outputs
                assert traffic >= 140 * n * K
                # scaled to a launch 5x as long
                g5 = bench._recorded(n, 5 * K, r["kernel"], r["launch"])
                assert g5["dram_bytes"] == 5 * traffic and g5["inst_executed_launch"] == 5 * int(r["inst_executed"])
        else:
            assert got is None


def test_traffic_lookup_refuses_other_workloads_and_launches():
    r = _records()[0]
    n, K = int(r["n_envs"]), int(r["steps_per_launch"])
    assert bench._recorded(n + 1, K, r["kernel"], r["launch"]) is None
    assert bench._recorded(n, K, "k_other", r["launch"]) is None
    assert bench._recorded(n, K, r["kernel"], "pipe:1w:7obs:map") is None


def test_launch_labels():
    base = dict(kernel="pipe", warps_per_block=16, warps_per_env=1, obs_warps=7, blocks_per_sm=0, order="map",
                segment=2048)
    assert bench.launch_label(base) == "pipe:16w:7obs:map:seg2048"
    assert bench.launch_label(dict(base, segment=0, order="index")) == "pipe:16w:7obs"
    assert bench.launch_label(dict(base, kernel="split", warps_per_env=3, segment=0, order="index")) == \
        "split:16w:3wpe"
    assert bench.launch_label(dict(base, kernel="queue", blocks_per_sm=2, order="cost", segment=0)) == \
        "queue:16w:2bps:cost"


def test_alu_roofline_arithmetic():
    # 1,772 samples per env-step, 1,024 envs x 10,000 steps in 10 ms at 2,070 MHz
    r = bench.roofline_alu(1772.0, 1024, 10000, 10.0, {"sm_mhz": 2070.0})
    peak = 152 * 128 * 2070e6 / 8 / 1e9
    assert r["bound"] == "alu" and abs(r["peak"] - peak) < 1e-9
    assert abs(r["achieved"] - 1772.0 * 1024 * 10000 / 0.01 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    # without the sample count (CPU leg skipped) there is no achieved value
    r = bench.roofline_alu(None, 1024, 10000, 10.0, None)
    assert r["achieved"] is None and r["frac"] is None and r["peak"] > 0


def test_streaming_view_arithmetic():
    """5,300 B per env-step (201^2/8 window bits + 250 B of SoA) at 1 G
    env-steps/s is 5,300 GB/s, against the measured HBM peak and the given
    L2 read peak."""
    v = bench.streaming_view(1e9, 153, {"peak_gbs": 20000.0})
    per = 201 * 201 / 8.0 + 250
    assert v["algorithmic_bytes_per_env_step"] == round(per)
    assert abs(v["achieved_gbs"] - per) < 1e-9
    assert abs(v["l2_frac"] - per / 20000.0) < 1e-12
    assert v["hbm_peak_gbs"] > 0 and abs(v["hbm_frac"] - per / v["hbm_peak_gbs"]) < 1e-12
    assert bench.streaming_view(1e9, 153, None)["l2_frac"] is None


def test_extras_selection_carries_the_ring_size():
    w = bench.ExtrasSel("qtc,full".split(","), 2)
    assert "qtc" in w and "full" in w and "step" not in w
    assert w.qtc_slots == 2
    assert not (w & {"qnet", "td"})
    assert bench.ExtrasSel(["step"]).qtc_slots == 64
