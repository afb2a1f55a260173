"""Host-side pieces of bench.py (no GPU): the source hash that ties committed
ncu records to the kernel they were taken on, the lookups of those records,
and the defaults the measurement contract depends on."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_and_whitespace_only(tmp_path):
    a = tmp_path / "a.cuh"
    b = tmp_path / "b.cuh"
    c = tmp_path / "c.cuh"
    a.write_text("int x = 1; // note\n/* block\n comment */ int y = x;\n")
    b.write_text("int  x = 1;\n\n\tint y = x; // another note\n")
    c.write_text("int x = 2; int y = x;\n")
    ha = bench._code_hash((str(a),))
    assert ha == bench._code_hash((str(b),))
    assert ha != bench._code_hash((str(c),))
    assert len(ha) == 16


def test_recorded_records_are_tied_to_their_configuration():
    t = bench.recorded_traffic("fp32", 384)
    assert t is None or t > 304 * 384 ** 3 * 0.9  # at least about the algorithmic bytes of a launch
    assert bench.recorded_traffic("fp32", 123) is None
    assert bench.recorded_traffic("fp16dev", 384) is None
    ops = bench.recorded_fp64_ops()
    assert ops is None or 100.0 < ops < 2000.0


def test_defaults_of_the_measurement_contract(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse_args()
    assert args.gpus == 1 and args.impl == "native"
    assert args.warmup >= 3 and args.steps >= 1
    assert args.size == 384 and args.stencil == 7
    cfg = bench.config_of(args)
    assert "384" in cfg["workload"]
    assert cfg["lattice"] == [384, 384, 384]
