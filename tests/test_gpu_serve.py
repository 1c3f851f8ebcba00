"""GPU tests of the serving loop (rfp_serve_*): results against the oracle,
the same result alone and in the mix (bit for bit), resident factors reused
by solve / invert requests, eviction under a small arena, and the error
statuses."""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

from gpu_util import factor_tolerance

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
srv_mod = pytest.importorskip("paper_0901_1696_gb300.serve")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

OPS, MODES = srv_mod, srv_mod
LAYOUTS = [("N", "L"), ("N", "U"), ("T", "L"), ("T", "U")]


def make_requests(specs, seed):
    """specs: (n, nrhs, mode, layout index) -> host inputs (pinned)."""
    reqs = []
    for k, (n, nrhs, mode, li) in enumerate(specs):
        t, u = LAYOUTS[li]
        A, rng = gen.spd_bbt(n, seed=seed * 1000 + k, return_rng=True)
        B = gen.rhs(n, nrhs, rng)
        arf = torch.from_numpy(oracle.pack(t, u, A)).pin_memory()
        Bh = torch.from_numpy(np.asfortranarray(B).ravel(order="F")).pin_memory()
        X = torch.zeros(n * nrhs, dtype=torch.float64).pin_memory()
        reqs.append(dict(id=k, n=n, nrhs=nrhs, mode=mode, t=t, u=u, A=A, B=B, arf=arf, Bh=Bh, X=X))
    return reqs


def submit(server, r, key=-1, op=srv_mod.OP_FACTOR_SOLVE):
    server.submit(r["id"], op, r["mode"], r["t"], r["u"], r["n"], r["nrhs"], arf=r["arf"],
                  B=r["Bh"], X=r["X"], key=key)


def check_solution(r):
    X = r["X"].numpy().reshape(r["nrhs"], r["n"]).T
    if r["mode"] == srv_mod.MODE_MIXED:
        assert oracle.solve_backward_error(r["A"], X, r["B"]) <= 1e-14
    else:
        fac, info = oracle.pftrf(r["t"], r["u"], r["n"], oracle.pack(r["t"], r["u"], r["A"]))
        ref = oracle.pftrs(r["t"], r["u"], r["n"], fac, r["B"])
        assert np.max(np.abs(X - ref)) <= factor_tolerance(r["n"]) * np.max(np.abs(ref))


SPECS = [(70, 3, 0, 0), (513, 2, 0, 1), (200, 8, 0, 2), (33, 1, 0, 3), (1500, 5, 0, 0),
         (450, 9, 0, 1), (300, 4, 1, 2), (1200, 16, 1, 3), (512, 8, 0, 2), (2100, 2, 0, 1),
         (64, 6, 0, 3), (900, 1, 1, 0), (128, 7, 0, 0), (257, 2, 0, 2)]


def test_serve_mix_matches_oracle_and_is_the_same_alone():
    reqs = make_requests(SPECS, seed=1)
    with srv_mod.Server(arena_bytes=2 << 30, streams=4, batch_max=64) as s:
        for r in reqs:
            submit(s, r)
        done = {c["id"]: c for c in s.wait(len(reqs))}
        st = s.stats()
    assert st["completed"] == len(reqs) and st["batches"] >= 1
    assert sum(c["batched"] for c in done.values()) >= 4   # the small FP64 requests
    mix = {}
    for r in reqs:
        c = done[r["id"]]
        assert c["status"] == 0, c
        assert c["t_submit"] <= c["t_start"] <= c["t_done"]
        check_solution(r)
        mix[r["id"]] = r["X"].numpy().copy()
    # each request alone, on a fresh server: bit-identical results
    for r in reqs:
        r["X"].zero_()
        with srv_mod.Server(arena_bytes=2 << 30, streams=4, batch_max=64) as s:
            submit(s, r)
            c = s.wait(1)[0]
        assert c["status"] == 0
        assert np.array_equal(r["X"].numpy(), mix[r["id"]]), r["id"]


def test_serve_resident_factor_solve_and_invert():
    r, = make_requests([(700, 3, 0, 1)], seed=2)
    with srv_mod.Server(arena_bytes=1 << 30, streams=2) as s:
        submit(s, r, key=42)
        c = s.wait(1)[0]
        assert c["status"] == 0 and c["cache_hit"] == 0
        check_solution(r)
        # a new right-hand side against the resident factor
        B2 = gen.rhs(r["n"], 4, seed=9)
        r2 = dict(r, id=1, nrhs=4, B=B2,
                  Bh=torch.from_numpy(np.asfortranarray(B2).ravel(order="F")).pin_memory(),
                  X=torch.zeros(r["n"] * 4, dtype=torch.float64).pin_memory())
        submit(s, r2, key=42, op=srv_mod.OP_SOLVE)
        c = s.wait(1)[0]
        assert c["status"] == 0 and c["cache_hit"] == 1
        check_solution(r2)
        # a factor+solve on the same key reuses the factor
        r["X"].zero_()
        submit(s, dict(r, id=2), key=42)
        c = s.wait(1)[0]
        assert c["status"] == 0 and c["cache_hit"] == 1
        check_solution(r)
        # the inverse in RFP from the resident factor
        nt = r["n"] * (r["n"] + 1) // 2
        Xi = torch.zeros(nt, dtype=torch.float64).pin_memory()
        s.submit(3, srv_mod.OP_INVERT, srv_mod.MODE_FP64, r["t"], r["u"], r["n"], 0, X=Xi, key=42)
        c = s.wait(1)[0]
        assert c["status"] == 0 and c["cache_hit"] == 1
        fac, _ = oracle.pftrf(r["t"], r["u"], r["n"], oracle.pack(r["t"], r["u"], r["A"]))
        ref, _ = oracle.pftri(r["t"], r["u"], r["n"], fac)
        assert np.max(np.abs(Xi.numpy() - ref)) <= factor_tolerance(r["n"]) * np.max(np.abs(ref))
        # unknown key
        s.submit(4, srv_mod.OP_SOLVE, srv_mod.MODE_FP64, r["t"], r["u"], r["n"], 4, B=r2["Bh"],
                 X=r2["X"], key=43)
        assert s.wait(1)[0]["status"] == srv_mod.E_NOKEY


def test_serve_small_arena_evicts_and_rejects_too_large():
    specs = [(1000, 2, 0, k % 4) for k in range(12)]      # 4 MB of RFP each
    reqs = make_requests(specs, seed=3)
    with srv_mod.Server(arena_bytes=24 << 20, streams=3, small_n=0) as s:
        for r in reqs:
            submit(s, r, key=100 + r["id"])
        done = s.wait(len(reqs))
        assert all(c["status"] == 0 for c in done)
        st = s.stats()
        assert st["evictions"] > 0 and st["cache_bytes"] <= 24 << 20
        for r in reqs:
            check_solution(r)
        big, = make_requests([(3000, 1, 0, 0)], seed=4)   # 36 MB of RFP > arena
        submit(s, dict(big, id=99))
        assert s.wait(1)[0]["status"] == srv_mod.E_TOOLARGE


def test_serve_not_spd_reports_pivot_and_drops_key():
    n = 600
    A = gen.spd_bbt(n, seed=5)
    A[400, 400] = -1.0
    t, u = "N", "L"
    arf = torch.from_numpy(oracle.pack(t, u, A)).pin_memory()
    B = torch.ones(n, dtype=torch.float64).pin_memory()
    X = torch.zeros(n, dtype=torch.float64).pin_memory()
    _, info = oracle.pftrf(t, u, n, oracle.pack(t, u, A))
    with srv_mod.Server(arena_bytes=256 << 20, streams=2) as s:
        s.submit(0, srv_mod.OP_FACTOR_SOLVE, srv_mod.MODE_FP64, t, u, n, 1, arf=arf, B=B, X=X, key=5)
        c = s.wait(1)[0]
        assert c["status"] == info > 0
        s.submit(1, srv_mod.OP_SOLVE, srv_mod.MODE_FP64, t, u, n, 1, B=B, X=X, key=5)
        assert s.wait(1)[0]["status"] == srv_mod.E_NOKEY


def test_serve_rejects_bad_requests():
    with srv_mod.Server(arena_bytes=64 << 20, streams=1) as s:
        B = torch.ones(4, dtype=torch.float64)
        with pytest.raises(rfp.RfpError) as e:
            s.submit(0, srv_mod.OP_FACTOR_SOLVE, 0, "C", "L", 4, 1, arf=B, B=B, X=B)
        assert e.value.status == -2
        with pytest.raises(rfp.RfpError):
            s.submit(0, srv_mod.OP_SOLVE, 0, "N", "L", 4, 1, B=B, X=B, key=-1)
        with pytest.raises(rfp.RfpError):
            s.submit(0, 7, 0, "N", "L", 4, 1, arf=B, B=B, X=B)
    with pytest.raises(rfp.RfpError):
        srv_mod.Server(arena_bytes=1024, streams=1)


def test_serve_two_long_requests_overlap_on_the_device():
    """Two long factor+solve requests submitted together run on two streams
    at once: their device intervals (CUDA events around each request's GPU
    work) intersect, and each result is the oracle's."""
    reqs = make_requests([(4000, 8, 0, 0), (4001, 8, 0, 3)], seed=6)
    with srv_mod.Server(arena_bytes=1 << 30, streams=4, small_n=0) as s:
        for r in reqs:
            submit(s, r)
        done = {c["id"]: c for c in s.wait(2)}
    a, b = done[0], done[1]
    for c in (a, b):
        assert c["status"] == 0 and c["batched"] == 0
        assert 0.0 < c["gpu_start_ms"] < c["gpu_end_ms"]
    assert max(a["gpu_start_ms"], b["gpu_start_ms"]) < min(a["gpu_end_ms"], b["gpu_end_ms"])
    for r in reqs:
        check_solution(r)


def test_serve_small_requests_with_many_rhs_and_mixed_mode_are_batched():
    """Factor+solve requests of order <= small_n with up to 32 right-hand
    sides, FP64 or mixed mode, go into batched launches; every result meets
    its mode's bar."""
    specs = [(100, 32, 0, 0), (257, 17, 1, 1), (512, 9, 1, 2), (64, 1, 0, 3), (300, 32, 1, 0)]
    reqs = make_requests(specs, seed=7)
    with srv_mod.Server(arena_bytes=1 << 30, streams=2, batch_max=64) as s:
        for r in reqs:
            submit(s, r)
        done = {c["id"]: c for c in s.wait(len(reqs))}
    for r in reqs:
        c = done[r["id"]]
        assert c["status"] == 0 and c["batched"] == 1, c
        assert c["gpu_start_ms"] <= c["gpu_end_ms"]
        check_solution(r)
