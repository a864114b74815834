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


# ------------------------------------------------ spectral comparison (Sec. 2, Table 2)

def test_spectral_table2():
    from tests.conftest import load_golden
    rows = load_golden("table2.txt")
    eps_p = rdct.spectral_error(rdct.VARIANT_ROUND)[0]
    eps_s = rdct.spectral_error(rdct.VARIANT_SDCT)[0]
    for row in rows[:-1]:
        m = int(row[0])
        assert round(eps_s[m], 2) == pytest.approx(float(row[1]), abs=1e-9), (m, eps_s[m])
        assert round(eps_p[m], 2) == pytest.approx(float(row[2]), abs=1e-9), (m, eps_p[m])
    sel = [1, 2, 3, 5, 6, 7]
    assert round(eps_s[sel].sum(), 2) == pytest.approx(float(rows[-1][1]))
    assert round(eps_p[sel].sum(), 2) == pytest.approx(float(rows[-1][2]))
    # Sec. 2: rows 0 and 4 of the proposed transform and of the signed DCT coincide with the DCT's
    assert eps_p[0] < 1e-20 and eps_p[4] < 1e-20 and eps_s[0] < 1e-20 and eps_s[4] < 1e-20


@pytest.mark.parametrize("name", ["round", "ceil", "sdct", "sdct_polar"])
def test_spectral_against_oracle_and_closed_form(name):
    eps, D, w = rdct.spectral_error(rdct.VARIANTS[name], 2001, want_curves=True)
    F, _ = orc.variant_matrices(name)
    np.testing.assert_allclose(D, orc.spectral_error(F, w), rtol=1e-10, atol=1e-14)
    # integral_0^pi |sum_n d_n e^{-jnw}|^2 dw = pi ||d||^2 for real taps d
    np.testing.assert_allclose(eps, np.pi * ((orc.dct_matrix() - F) ** 2).sum(axis=1), rtol=1e-9, atol=1e-15)


def test_spectral_rejects():
    with pytest.raises(rdct.RdctError):
        rdct.spectral_error(rdct.VARIANT_ROUND, 2000)
    with pytest.raises(rdct.RdctError):
        rdct.spectral_error(rdct.VARIANT_FLOOR)
