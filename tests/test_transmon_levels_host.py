"""The operator builder's transmon eigenbasis (host side, before the C-ABI) agrees
with the oracle's independent construction: same energies, same charge matrix."""
import numpy as np
import pytest

from oracle import systems as OS
from paper_2605_27515_gb300 import systems

EC = 2 * np.pi * 0.28


@pytest.mark.parametrize("ej_over_ec,K,n_cut", [(50.0, 32, 500), (50.0, 64, 500), (10.0, 16, 80), (0.0, 9, 20)])
def test_builder_matches_oracle(ej_over_ec, K, n_cut):
    ej = ej_over_ec * EC
    E_b, nt_b = systems.transmon_levels(EC, ej, K, n_cut)
    E_o, nt_o, _ = OS.transmon_eigenbasis(EC, ej, K, n_cut=n_cut)
    scale = max(1.0, np.abs(E_o).max())
    np.testing.assert_allclose(E_b, E_o, atol=1e-11 * scale)
    np.testing.assert_allclose(nt_b, nt_o, atol=1e-9)
