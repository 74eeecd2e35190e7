"""The benchmark's bookkeeping (no GPU): algorithmic bytes and flops per pass, the variant
key that selects a committed ncu record, and the per-grid-point figures quoted with them."""
import json
import os

import pytest

bench = pytest.importorskip("bench")


@pytest.mark.parametrize("n", [64, 512, 4096, 8192])
def test_algorithmic_bytes_count_each_input_and_output_once(n):
    H, NK = n // 4 + 1, n // 2 + 1
    for elt in (4, 8):
        b = bench.algorithmic_bytes(n, elt)
        c = 2 * elt                                    # one complex value
        assert b["row_pass"] == 3 * H * n * c + n * n * elt + 3 * H * n * c
        assert b["col_pass"] == 3 * H * n * c + 2 * H * NK * c + 3 * H * n * c
    b = bench.algorithmic_bytes(n, 4)
    per_point = (b["row_pass"] + b["col_pass"]) / (n * n)
    if n >= 512:                                       # the +1 column matters on small grids
        assert 29.0 < per_point < 31.5                 # ~30 B per grid-point-step in FP32


def test_algorithmic_bytes_and_flops_at_512():
    b = bench.algorithmic_bytes(512, 4)
    assert b["row_pass"] == 4218880
    f = bench.algorithmic_flops(512)
    assert abs((f["row_pass"] + f["col_pass"]) / 512 ** 2 - 234) < 1.0
    assert abs(f["row_pass"] / 1e6 - 42.6) < 0.1


def test_plan_variant_keys_match_the_record_layout():
    plan = {"rows_per_block": 4, "row_points_per_thread": 16, "col_points_per_thread": 8, "row_cluster": 1}
    assert bench.plan_variant("row_pass", plan) == [4, 16]
    assert bench.plan_variant("col_pass", plan) == [8]
    assert bench.plan_variant("row_pass", dict(plan, rows_per_block=1, row_cluster=2)) == [1, 16, 2]
    recs = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["records"]
    for key, entries in recs.items():
        kernel, n, prec = key.split(":")
        assert kernel in ("row_pass", "col_pass") and int(n) > 0 and prec in ("32", "64")
        for e in entries:
            assert e["dram_bytes_per_launch"] > 0 and len(e["variant"]) in ((1,) if kernel == "col_pass" else (2, 3))


def test_oracle_replicas_time_every_process():
    """The all-core CPU baseline: independent oracle processes (spawned), each timed over its
    own copy of the workload; the aggregate is the sum of their rates."""
    rate, P, steps, wall = bench.oracle_replicas("circle64_fp64", 10, procs=2, warm_steps=1, timed_steps=5)
    assert P == 2 and steps == [5, 5] and wall > 0
    assert rate > 0
