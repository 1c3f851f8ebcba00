"""CPU checks of the input recipes that the bench and the serving workload
rely on (rfp_inputs): symmetry, spectrum endpoints and determinism."""
import numpy as np
import pytest

import rfp_inputs as gen

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,kappa", [(1, 10.0), (2, 1e3), (97, 1e6), (256, 1e1)])
def test_reflector_matrices_have_the_prescribed_spectrum(n, kappa):
    A = gen.spd_reflectors(n, seed=n, kappa=kappa, device="cpu").numpy()
    assert np.array_equal(A, A.T)
    w = np.linalg.eigvalsh(A)
    assert abs(w[0] - 1.0) < 1e-9 * kappa
    if n > 1:
        assert abs(w[-1] - kappa) < 1e-9 * kappa
    assert np.all(w > 0.5)
    B = gen.spd_reflectors(n, seed=n, kappa=kappa, device="cpu").numpy()
    assert np.array_equal(A, B)                     # a pure function of its arguments
    if n > 2:
        assert np.count_nonzero(A) == n * n         # dense: every entry mixed
