"""Work counts used to turn times into rates.

PFTRF = n^3/3 flops: the paper's own tables fix this convention (rate x time
= n^3/3 in Table "ibmpar", e.g. 2551 Mflop/s x 16.34 s at n = 5000).  PFTRS =
2 n^2 nrhs and PFTRI = 2 n^3/3 follow the LAPACK convention (the paper does
not state them).  Pack / unpack move the stored triangle once each way:
2 * n(n+1)/2 elements.
"""


def pftrf_flops(n: int) -> float:
    return n ** 3 / 3.0


def pftrs_flops(n: int, nrhs: int) -> float:
    return 2.0 * n * n * nrhs


def pftri_flops(n: int) -> float:
    return 2.0 * n ** 3 / 3.0


def pack_bytes(n: int, elem_size: int = 8) -> int:
    return 2 * (n * (n + 1) // 2) * elem_size
