"""Host-side helpers of the batched path (no GPU): the entry table builder,
the n-bucket map and the tuning cache."""
import json

import numpy as np
import pytest

from paper_0901_1696_gb300 import batched as bt


def test_make_entries_offsets_and_lengths():
    ns, nrhs = [0, 5, 32, 512, 7], [3, 1, 8, 2, 0]
    e, arf_len, b_len = bt.make_entries(ns, ["N", "T", "N", "T", "N"], ["L", "U", "U", "L", "L"],
                                       nrhs)
    nt = [n * (n + 1) // 2 for n in ns]
    assert list(e["arf"]) == [0, 0, 15, 15 + 528, 15 + 528 + 131328]
    assert arf_len == sum(nt)
    assert list(e["b"]) == [0, 0, 5, 5 + 256, 5 + 256 + 1024]
    assert b_len == sum(n * r for n, r in zip(ns, nrhs))
    assert list(e["ldb"]) == [1, 5, 32, 512, 7]
    assert e["transr"][1] == b"T" and e["uplo"][2] == b"U"
    assert list(e["nb"]) == [0] * 5
    # every matrix's arrays stay inside the buffers, as rfp_batch_plan checks
    for k in range(len(ns)):
        assert e["arf"][k] + nt[k] <= arf_len
        if ns[k] and nrhs[k]:
            assert e["b"][k] + (nrhs[k] - 1) * e["ldb"][k] + ns[k] <= b_len


def test_bucket_boundaries():
    assert bt.bucket_of(0) == 0 and bt.bucket_of(64) == 0 and bt.bucket_of(65) == 1
    assert bt.bucket_of(512) == len(bt.BUCKETS) - 1
    with pytest.raises(ValueError):
        bt.bucket_of(513)


def test_tuning_cache_round_trip_and_fill(tmp_path):
    path = tmp_path / "tune.json"
    c = bt.TuningCache(str(path))
    assert c.get("GPU", "f64") is None
    e, _, _ = bt.make_entries([10, 100, 300, 500], ["N", "T", "N", "T"], ["L"] * 4, [1] * 4)
    assert not c.fill_nb(e, "GPU", "f64")
    table = {"N": [16, 16, 32, 32, 32, 32, 16, 32], "T": [32, 16, 16, 16, 16, 16, 16, 16]}
    c.put("GPU", "f64", table)
    assert json.loads(path.read_text())["GPU"]["f64"] == table
    c2 = bt.TuningCache(str(path))
    assert c2.fill_nb(e, "GPU", "f64")
    assert list(e["nb"]) == [16, 16, 32, 16]
