"""Host-side measurement helpers of bench.py (no GPU): the DRAM traffic taken
from the committed ncu summary only while the kernel's source files are the
ones it was captured on, and the tuner-gain summary."""
import json
import os

import pytest

import bench


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    root = tmp_path
    csrc = root / "paper_2307_08606_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    (csrc / "k.cu").write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.source_sha(["k.cu"])
    entry = {"kernel": "k", "files": ["k.cu"], "source_sha": sha, "dram_bytes_per_launch": 1234}
    (root / "profiles" / "traffic.json").write_text(json.dumps({"kernels": {"fwd": entry}}))
    assert bench.traffic_for("fwd") == 1234.0
    assert bench.traffic_for("other") is None
    (csrc / "k.cu").write_text("kernel v2")          # the kernel changed since the capture
    assert bench.traffic_for("fwd") is None


def test_committed_traffic_summary_names_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for name, e in t["kernels"].items():
        assert e["dram_bytes_per_launch"] > 0, name
        for fn in e["files"]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2307_08606_gb300", "csrc", fn)), fn


def test_tuning_gain_is_relative_to_the_default_splits():
    t = [{"forward": {2: 1.0, 4: 0.8}, "adjoint": {1: 2.0, 2: 1.5},
          "forward_default": 2, "adjoint_default": 1, "forward_splits": 4, "adjoint_splits": 2}]
    assert bench._tuning_gain(t) == pytest.approx((3.0 - 2.3) / 3.0)
    t[0]["forward_splits"], t[0]["adjoint_splits"] = 2, 1
    assert bench._tuning_gain(t) == 0.0


def test_gpus_flag_starts_that_many_ranks(monkeypatch):
    """`--gpus N` without a launcher re-runs the bench under
    torch.distributed.run with N processes on 127.0.0.1; a launcher that
    started a different number of ranks than --gpus is refused."""
    calls = []
    monkeypatch.setattr(bench.subprocess, "call", lambda cmd: calls.append(cmd) or 0)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench.sys, "argv", ["bench.py", "--gpus", "4", "--steps", "2"])
    assert bench.main() == 0
    cmd = calls[0]
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "127.0.0.1" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "2"] and cmd[-5].endswith("bench.py")
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(SystemExit, match="--gpus 4 but the launcher started 2 ranks"):
        bench.main()


def test_factor_order_follows_the_smaller_gram():
    """The x-update factor of Eq. 3 is 2KM x 2KM (Woodbury) when N > 2KM and
    N x N (primal) otherwise: the bytes the batched factor apply streams."""
    import scenegen
    g = scenegen.GEOMS["resolved_128"]              # KM = 16384, N = 128^2: primal
    assert bench._factor_order(g) == g.N == 16384
    p = scenegen.GEOMS["paper_scale"]               # KM = 2048, N = 128^2: Woodbury
    assert bench._factor_order(p) == 2 * p.KM == 4096


def test_the_committed_traffic_matches_the_current_kernels():
    """profiles/traffic.json was captured on the current sources of the
    single-scene kernels, so the bench reports their DRAM traffic."""
    for k in ("forward", "adjoint_update", "spd_woodbury"):
        assert bench.traffic_for(k) is not None, k
