"""GPU tests of the batched path (rfp_batch_plan + rfp_{d,s}pfsv_batched).

Each matrix of a batch of uneven orders (0 to 512) and mixed layouts is
compared with the oracle's own factorization and solve, element by element
within gpu_util.factor_tolerance, and its info with the oracle's.  The
results must be identical bit for bit (a) when the launch is captured in a
CUDA graph and replayed and (b) when a matrix is solved alone instead of in
the mix: the per-matrix work never depends on the other matrices.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

from gpu_util import EPS32, factor_tolerance

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

LAYOUTS8 = [(t, u) for t in "NT" for u in "LU"]


def make_batch(count, seed, n_max=512, fail_every=0):
    """Host inputs: entries, packed A, B, and the per-matrix data for checks."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(0, n_max + 1, count)
    ns[: min(count, 8)] = [0, 1, 2, 31, 32, 33, 511, 512][: min(count, 8)]
    entries = np.zeros(count, dtype=rfp.batch_entry_dtype())
    mats, arf_parts, b_parts, fails = [], [], [], []
    arf_off = b_off = 0
    for k, n in enumerate(ns):
        n = int(n)
        transr, uplo = LAYOUTS8[rng.integers(0, 4)]
        nrhs = int(rng.integers(0, 33))   # up to 32: solved in passes of 8 columns
        A, r2 = gen.spd_bbt(n, seed=1000 + seed * 10000 + k, return_rng=True)
        fail = 0
        if fail_every and k % fail_every == fail_every - 1 and n > 2:
            j = int(rng.integers(0, n))
            A = A.copy()
            A[j, j] = -1.0 - np.sum(np.abs(A[j]))            # pivot j is <= 0 for sure
            fail = -1                                        # index from the oracle below
        B = gen.rhs(n, nrhs, r2) if nrhs else np.zeros((n, 0))
        arf = oracle.pack(transr, uplo, A)
        entries[k] = (n, arf_off, b_off, nrhs, max(n, 1), transr.encode(), uplo.encode(),
                      [0, 16, 24, 32][k % 4], 0)
        mats.append(dict(n=n, A=A, B=B, transr=transr, uplo=uplo, nrhs=nrhs, arf_off=arf_off,
                         b_off=b_off, fail=fail))
        arf_parts.append(arf)
        b_parts.append(B.ravel(order="F"))
        arf_off += arf.size
        b_off += B.size
    arf_all = np.concatenate(arf_parts) if arf_parts else np.zeros(0)
    b_all = np.concatenate(b_parts) if b_parts else np.zeros(0)
    return entries, arf_all, b_all, mats


def run_batch(entries, arf_all, b_all, dtype=torch.float64, stream=None):
    count = len(entries)
    plan = torch.empty(rfp.rfp_batch_plan_bytes(count), dtype=torch.uint8, device="cuda")
    rfp.rfp_batch_plan(count, entries, arf_all.size, b_all.size, plan, plan.numel())
    d_arf = torch.from_numpy(arf_all).to(dtype).cuda() if arf_all.size else \
        torch.zeros(1, dtype=dtype, device="cuda")          # the library wants a real pointer
    d_b = torch.from_numpy(b_all).to(dtype).cuda() if b_all.size else \
        torch.zeros(1, dtype=dtype, device="cuda")
    info = torch.full((count,), -7, dtype=torch.int32, device="cuda")
    fn = rfp.rfp_dpfsv_batched if dtype == torch.float64 else rfp.rfp_spfsv_batched
    fn(count, plan, d_arf, d_b, info)
    torch.cuda.synchronize()
    return plan, d_arf, d_b, info


def check_results(mats, arf_out, b_out, info_out, eps=None):
    for k, m in enumerate(mats):
        n, t, u = m["n"], m["transr"], m["uplo"]
        nt = n * (n + 1) // 2
        ref, ref_info = oracle.pftrf(t, u, n, oracle.pack(t, u, m["A"]))
        assert info_out[k] == ref_info, (k, n, info_out[k], ref_info)
        if ref_info:
            continue
        fac = arf_out[m["arf_off"]: m["arf_off"] + nt]
        tol = factor_tolerance(n) if eps is None else factor_tolerance(n, eps=eps)
        if n:
            assert np.max(np.abs(fac - ref)) <= tol * np.max(np.abs(ref)), (k, n)
        if m["nrhs"] and n:
            X = b_out[m["b_off"]: m["b_off"] + n * m["nrhs"]].reshape(m["nrhs"], n).T
            Xr = oracle.pftrs(t, u, n, ref, m["B"])
            assert np.max(np.abs(X - Xr)) <= tol * np.max(np.abs(Xr)), (k, n)


def test_batched_fp64_uneven_mixed_layouts():
    entries, arf_all, b_all, mats = make_batch(300, seed=1, fail_every=97)
    _, d_arf, d_b, info = run_batch(entries, arf_all, b_all)
    assert sum(1 for m in mats if m["fail"]) >= 2
    check_results(mats, d_arf.cpu().numpy(), d_b.cpu().numpy(), info.cpu().numpy())


def test_batched_fp32():
    entries, arf_all, b_all, mats = make_batch(120, seed=2)
    for m in mats:                                  # compare in the precision actually stored
        m["A"] = m["A"].astype(np.float32).astype(np.float64)
        m["B"] = m["B"].astype(np.float32).astype(np.float64)
    arf32 = np.concatenate([oracle.pack(m["transr"], m["uplo"], m["A"]) for m in mats])
    b32 = np.concatenate([m["B"].ravel(order="F") for m in mats])
    _, d_arf, d_b, info = run_batch(entries, arf32, b32, dtype=torch.float32)
    check_results(mats, d_arf.cpu().numpy().astype(np.float64), d_b.cpu().numpy().astype(np.float64),
                  info.cpu().numpy(), eps=EPS32)


def test_batched_graph_capture_and_alone_vs_mix_bit_identical():
    entries, arf_all, b_all, mats = make_batch(64, seed=3)
    count = len(entries)
    plan, d_arf, d_b, info = run_batch(entries, arf_all, b_all)
    eager_arf, eager_b = d_arf.cpu().numpy(), d_b.cpu().numpy()
    # CUDA graph: capture once, replay on fresh inputs
    g_arf = torch.from_numpy(arf_all).cuda()
    g_b = torch.from_numpy(b_all).cuda()
    g_info = torch.zeros(count, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rfp.rfp_dpfsv_batched(count, plan, g_arf, g_b, g_info, stream=s)
    for _ in range(2):
        g_arf.copy_(torch.from_numpy(arf_all))
        g_b.copy_(torch.from_numpy(b_all))
        graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(g_arf.cpu().numpy(), eager_arf)
    assert np.array_equal(g_b.cpu().numpy(), eager_b)
    # alone vs in the mix
    for k in [0, 7, 20, 41, 63]:
        m = mats[k]
        nt = m["n"] * (m["n"] + 1) // 2
        one = entries[k:k + 1].copy()
        one["arf"], one["b"] = 0, 0
        a1 = arf_all[m["arf_off"]: m["arf_off"] + nt]
        b1 = b_all[m["b_off"]: m["b_off"] + m["n"] * m["nrhs"]]
        _, d1, db1, _ = run_batch(one, a1, b1)
        assert np.array_equal(d1.cpu().numpy()[:nt], eager_arf[m["arf_off"]: m["arf_off"] + nt])
        if m["nrhs"] and m["n"]:
            assert np.array_equal(db1.cpu().numpy()[: b1.size],
                                  eager_b[m["b_off"]: m["b_off"] + b1.size])


def test_autotune_small_writes_cache(tmp_path):
    """The autotuner times both panel widths per bucket and TRANSR (tiny
    batches here) and stores a complete table that fill_nb can apply."""
    from paper_0901_1696_gb300 import batched as bt
    cache = bt.TuningCache(str(tmp_path / "tune.json"))
    table = bt.autotune("f64", count=4, reps=1, cache=cache)
    assert set(table) == {"N", "T"}
    for t in "NT":
        assert len(table[t]) == len(bt.BUCKETS) and set(table[t]) <= {16, 24, 32}
    gpu = torch.cuda.get_device_properties(0).name
    assert bt.TuningCache(str(tmp_path / "tune.json")).get(gpu, "f64") == table
    e, _, _ = bt.make_entries([40, 400], ["N", "T"], ["L", "U"], [1, 2])
    assert cache.fill_nb(e, gpu, "f64") and set(e["nb"]) <= {16, 24, 32}


def test_plan_rejects_more_than_32_right_hand_sides():
    entries = np.zeros(2, dtype=rfp.batch_entry_dtype())
    for k, r in enumerate((32, 33)):
        entries[k] = (10, 55 * k, 10 * 32 * k, r, 10, b"N", b"L", 16, 0)
    plan = torch.empty(rfp.rfp_batch_plan_bytes(2), dtype=torch.uint8, device="cuda")
    with pytest.raises(rfp.RfpError) as e:
        rfp.rfp_batch_plan(2, entries, 110, 10 * 32 + 10 * 33, plan, plan.numel())
    assert e.value.status == -2 and "entry 1" in str(e.value)
