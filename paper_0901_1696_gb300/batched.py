"""Host-side helpers of the batched path (rfp_batch_plan / rfp_{d,s}pfsv_batched).

* ``make_entries``: the rfp_batch_entry_t table for a list of matrices laid
  out back to back in one RFP buffer and one right-hand-side buffer.
* ``TuningCache``: the panel width (nb = 16, 24 or 32) chosen per n-bucket,
  TRANSR and precision, kept in a JSON file per GPU model.
* ``autotune``: measures every panel width on synthetic batches of each
  bucket (one graph-captured launch per batch, as the batched call is used)
  and stores the fastest.

The tuning only chooses among launch variants of the same kernel; results
are identical in exact arithmetic and the per-matrix work never depends on
the other matrices.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import binding as rfp

BUCKETS = (64, 128, 192, 256, 320, 384, 448, 512)   # upper ends of the n-buckets
PANEL_WIDTHS = (16, 24, 32)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "batched_tuning.json")
# Tables measured by `autotune` on each listed GPU model and shipped with the
# package, so that a fresh machine of that model needs no tuning run.
SHIPPED_TABLES = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                              "batched_tuning_shipped.json")


def bucket_of(n: int) -> int:
    for b, hi in enumerate(BUCKETS):
        if n <= hi:
            return b
    raise ValueError(f"order {n} exceeds the batched path's maximum {BUCKETS[-1]}")


def make_entries(ns, transrs, uplos, nrhss, nb=None):
    """Entries for matrices stored back to back: matrix k's RFP array at the
    running offset sum_{l<k} n_l (n_l + 1) / 2 and its right-hand sides
    (column-major, ldb = max(1, n_k)) at sum_{l<k} n_l nrhs_l.  Returns
    (entries, arf_len, b_len)."""
    count = len(ns)
    e = np.zeros(count, dtype=rfp.batch_entry_dtype())
    ns = np.asarray(ns, dtype=np.int64)
    nrhss = np.asarray(nrhss, dtype=np.int64)
    nt = ns * (ns + 1) // 2
    e["n"] = ns
    e["arf"] = np.concatenate([[0], np.cumsum(nt)[:-1]]) if count else []
    e["b"] = np.concatenate([[0], np.cumsum(ns * nrhss)[:-1]]) if count else []
    e["nrhs"] = nrhss
    e["ldb"] = np.maximum(ns, 1)
    e["transr"] = [t.encode() for t in transrs]
    e["uplo"] = [u.encode() for u in uplos]
    e["nb"] = 0 if nb is None else nb
    return e, int(nt.sum()), int((ns * nrhss).sum())


def _shipped() -> dict:
    if os.path.exists(SHIPPED_TABLES):
        with open(SHIPPED_TABLES) as f:
            return json.load(f)
    return {}


class TuningCache:
    """{gpu name: {"f64" | "f32": {"N" | "T": [nb per bucket]}}} in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("RFP_BATCHED_TUNING", DEFAULT_CACHE)
        self.data = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.data = json.load(f)

    def get(self, gpu: str, prec: str):
        """The table tuned on this machine, else the shipped one, else None."""
        return self.data.get(gpu, {}).get(prec) or _shipped().get(gpu, {}).get(prec)

    def source(self, gpu: str, prec: str):
        if self.data.get(gpu, {}).get(prec):
            return "tuned on this machine"
        if _shipped().get(gpu, {}).get(prec):
            return "shipped table for this GPU model"
        return None

    def put(self, gpu: str, prec: str, table: dict):
        self.data.setdefault(gpu, {})[prec] = table
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def fill_nb(self, entries, gpu: str, prec: str) -> bool:
        """Set entries["nb"] from the table; False (nb left as is) if none."""
        table = self.get(gpu, prec)
        if not table:
            return False
        for k in range(len(entries)):
            t = entries["transr"][k].decode().upper()
            entries["nb"][k] = table[t][bucket_of(int(entries["n"][k]))]
        return True


def _synthetic_batch(torch, lib, ns, transr, dtype, seed):
    """Device RFP arrays of diagonally dominant SPD matrices A = S + n I (S
    symmetric, entries in [-1, 1)), packed with the library's own pack."""
    dev = torch.device("cuda", torch.cuda.current_device())
    entries, arf_len, b_len = make_entries(ns, [transr] * len(ns), ["L"] * len(ns),
                                           [1] * len(ns))
    arf = torch.empty(max(arf_len, 1), dtype=dtype, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    pack = lib.rfp_dpack if dtype == torch.float64 else lib.rfp_spack
    for k, n in enumerate(ns):
        S = torch.rand(n, n, dtype=dtype, device=dev, generator=g) * 2 - 1
        A = (S + S.T) * 0.5 + n * torch.eye(n, dtype=dtype, device=dev)
        pack(transr, "L", n, A, n, arf[int(entries["arf"][k]):])
    B = torch.ones(max(b_len, 1), dtype=dtype, device=dev)
    return entries, arf, B


def time_batch(torch, lib, entries, arf, B, dtype, reps=3):
    """Median device time (ms) of one graph-captured batched call, with the
    inputs restored before every replay (restores not timed)."""
    dev = arf.device
    count = len(entries)
    plan = torch.empty(lib.rfp_batch_plan_bytes(count), dtype=torch.uint8, device=dev)
    lib.rfp_batch_plan(count, entries, arf.numel(), B.numel(), plan, plan.numel())
    work_a, work_b = arf.clone(), B.clone()
    info = torch.zeros(count, dtype=torch.int32, device=dev)
    fn = lib.rfp_dpfsv_batched if dtype == torch.float64 else lib.rfp_spfsv_batched
    s = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fn(count, plan, work_a, work_b, info, stream=s)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for _ in range(reps):
        with torch.cuda.stream(s):
            work_a.copy_(arf)
            work_b.copy_(B)
            ev[0].record(s)
            graph.replay()
            ev[1].record(s)
        torch.cuda.synchronize(dev)
        times.append(ev[0].elapsed_time(ev[1]))
    if int(info.abs().sum().item()) != 0:
        raise RuntimeError("batched tuning matrices failed to factor")
    return float(np.median(times)), work_a, work_b, info


def autotune(prec: str = "f64", count: int | None = None, reps: int = 3, cache=None,
             seed: int = 0):
    """Measure nb = 16, 24 and 32 for every n-bucket and TRANSR on batches of
    `count` matrices (default: two per SM) with n uniform in the bucket;
    store and return {"N": [...], "T": [...]}."""
    import torch
    lib = rfp.library()
    dtype = torch.float64 if prec == "f64" else torch.float32
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    count = count or 2 * props.multi_processor_count
    rng = np.random.default_rng(seed)
    table = {}
    for transr in ("N", "T"):
        best = []
        for b, hi in enumerate(BUCKETS):
            lo = BUCKETS[b - 1] + 1 if b else 1
            ns = [int(x) for x in rng.integers(lo, hi + 1, count)]
            entries, arf, B = _synthetic_batch(torch, lib, ns, transr, dtype, seed + b)
            t = {}
            for nb in PANEL_WIDTHS:
                entries["nb"] = nb
                t[nb] = time_batch(torch, lib, entries, arf, B, dtype, reps)[0]
            best.append(min(t, key=t.get))
        table[transr] = best
    cache = cache or TuningCache()
    cache.put(props.name, prec, table)
    return table
