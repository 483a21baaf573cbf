"""Host logic of bench.py that needs no GPU: the DRAM traffic recorded by an
ncu capture is reported only for the workload it was captured on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1905_11071_gb300 import synth  # noqa: E402


def _args(prec="bf16x3", backward="traj"):
    return type("A", (), {"prec": prec, "oista_prec": "bf16x3", "backward": backward})()


def test_traffic_record_names_its_workload():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        doc = json.load(f)
    assert set(bench.TRAFFIC_KEYS) <= set(doc["config"])
    assert set(doc["parts"]) == {"gram", "slista_fwd", "objective", "slista_bwd"}


@pytest.mark.parametrize("N,T,prec,backward", [(1000, 40, "bf16x3", "traj"), (10000, 20, "bf16x3", "traj"),
                                                (10000, 40, "fp32", "traj"), (10000, 40, "bf16x3", "ckpt")])
def test_traffic_withheld_for_another_workload(N, T, prec, backward):
    cfg = bench.arm_config(synth.slista_64x256(N=N, T=T), _args(prec, backward), 1)
    for part in ("gram", "slista_fwd", "objective", "slista_bwd"):
        assert bench.recorded_traffic(part, cfg) is None
