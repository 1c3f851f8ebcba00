"""ctypes wrapper of the serving loop (rfp_serve_* in include/rfp.h).

Argument marshalling only: the scheduler, the arena, the factor cache and
the batching all run in the library.  Host arrays may be numpy arrays,
torch tensors (pinned CPU tensors make the copies asynchronous) or raw
addresses; they must stay alive until their request's completion is polled.
"""
from __future__ import annotations

import ctypes

from . import binding as rfp

OP_FACTOR_SOLVE, OP_SOLVE, OP_INVERT = 0, 1, 2
MODE_FP64, MODE_MIXED = 0, 1
E_TOOLARGE, E_NOKEY, E_NOCONV, E_CUDA = -101, -102, -103, -104


class ServeConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("streams", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("small_n", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("batch_nb", (ctypes.c_int16 * 8) * 2)]


class ServeRequest(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("key", ctypes.c_int64), ("n", ctypes.c_int64),
                ("nrhs", ctypes.c_int32), ("op", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("transr", ctypes.c_char), ("uplo", ctypes.c_char), ("reserved", ctypes.c_int16),
                ("arf", ctypes.c_void_p), ("B", ctypes.c_void_p), ("X", ctypes.c_void_p)]


class ServeCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("cache_hit", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("backward_error", ctypes.c_double), ("gpu_start_ms", ctypes.c_double),
                ("gpu_end_ms", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("cache_hits", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("cache_entries", ctypes.c_int64), ("cache_bytes", ctypes.c_size_t),
                ("arena_in_use", ctypes.c_size_t), ("arena_capacity", ctypes.c_size_t)]


def _sigs(lib):
    p = ctypes.c_void_p
    lib.rfp_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(p)]
    lib.rfp_serve_submit.argtypes = [p, ctypes.POINTER(ServeRequest)]
    lib.rfp_serve_poll.argtypes = [p, ctypes.POINTER(ServeCompletion), ctypes.c_int, ctypes.c_double]
    lib.rfp_serve_stats.argtypes = [p, ctypes.POINTER(ServeStats)]
    lib.rfp_serve_destroy.argtypes = [p]
    for f in ("rfp_serve_create", "rfp_serve_submit", "rfp_serve_poll", "rfp_serve_stats",
              "rfp_serve_destroy"):
        getattr(lib, f).restype = ctypes.c_int


class Server:
    """One serving loop on the current CUDA device."""

    def __init__(self, arena_bytes: int, streams: int = 4, batch_max: int = 1024,
                 small_n: int = 512, max_iter: int = 30, tol: float = 1e-15, batch_nb=None,
                 library: rfp.Library | None = None):
        self.lib = (library or rfp.library()).lib
        _sigs(self.lib)
        cfg = ServeConfig(arena_bytes=arena_bytes, streams=streams, batch_max=batch_max,
                          small_n=small_n, max_iter=max_iter, tol=tol)
        if batch_nb is not None:
            for t in range(2):
                for b in range(8):
                    cfg.batch_nb[t][b] = int(batch_nb[t][b])
        h = ctypes.c_void_p()
        rc = self.lib.rfp_serve_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise rfp.RfpError("rfp_serve_create", rc)
        self.handle = h
        self._buf = (ServeCompletion * 1024)()

    def submit(self, id: int, op: int, mode: int, transr: str, uplo: str, n: int, nrhs: int,
               arf=None, B=None, X=None, key: int = -1):
        r = ServeRequest(id=id, key=key, n=n, nrhs=nrhs, op=op, mode=mode,
                         transr=transr.encode(), uplo=uplo.encode(), arf=rfp._addr(arf),
                         B=rfp._addr(B), X=rfp._addr(X))
        rc = self.lib.rfp_serve_submit(self.handle, ctypes.byref(r))
        if rc != 0:
            raise rfp.RfpError("rfp_serve_submit", rc)

    def poll(self, max_items: int = 1024, timeout: float = 0.05) -> list[dict]:
        k = self.lib.rfp_serve_poll(self.handle, self._buf, min(max_items, 1024), timeout)
        if k < 0:
            raise rfp.RfpError("rfp_serve_poll", k)
        return [{f: getattr(self._buf[i], f) for f, _ in ServeCompletion._fields_}
                for i in range(k)]

    def wait(self, count: int, timeout: float = 600.0) -> list[dict]:
        """Poll until `count` completions have arrived."""
        import time
        out, t0 = [], time.time()
        while len(out) < count:
            out += self.poll(timeout=0.05)
            if time.time() - t0 > timeout:
                raise TimeoutError(f"{len(out)} of {count} completions after {timeout} s")
        return out

    def stats(self) -> dict:
        s = ServeStats()
        self.lib.rfp_serve_stats(self.handle, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def close(self):
        if self.handle:
            self.lib.rfp_serve_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
