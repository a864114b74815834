"""The library's host-side matrices of the other transforms (signed DCT, ceil / floor
variants) against the oracle's, which are built independently (numpy eigh / inv vs the
library's Jacobi / Gauss-Jordan).  Pure host code: runs without a GPU."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct


@pytest.mark.parametrize("name", ["round", "ceil", "sdct", "sdct_polar"])
def test_variant_matrices_match_oracle(name):
    F, G = rdct.variant_matrices(rdct.VARIANTS[name])
    Fo, Go = orc.variant_matrices(name)
    np.testing.assert_allclose(F, Fo, atol=1e-13)
    np.testing.assert_allclose(G, Go, atol=1e-13)
    np.testing.assert_allclose(G @ F, np.eye(8), atol=1e-13)


def test_floor_variant_refused():
    with pytest.raises(rdct.RdctError) as e:
        rdct.variant_matrices(rdct.VARIANT_FLOOR)
    assert e.value.status == 1
    with pytest.raises(rdct.RdctError):
        rdct.variant_matrices(17)
