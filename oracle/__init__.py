"""Plain CPU FP64 oracle for RFPF Cholesky (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing from it.  See ``rfp_oracle.c`` for the passages each
function follows.
"""
from .oracle import (  # noqa: F401
    OracleError,
    ar_shape,
    build,
    factor_residual,
    inverse_residual,
    lib_path,
    pack,
    pftrf,
    pftri,
    pftrs,
    potrf_full,
    solve_backward_error,
    split,
    unpack,
)
from .lapack_surface import (  # noqa: F401
    full_to_tp,
    lansf,
    sfrk,
    tfsm,
    tfttp,
    tftri,
    tp_index,
    tp_to_full,
    tpttf,
    tri_inverse,
)
