"""Porosity labels of the meshwork permeability (Kozeny-Carman fit of
Tab. 5): every printed (porosity, permeability) pair, the inverse, and the
limits of the relation."""
import os

import pytest

from paper_2102_12663_gb300.calibrate import (KOZENY_CARMAN_C, permeability_from_porosity,
                                              porosity_from_permeability)

HERE = os.path.dirname(os.path.abspath(__file__))


def tab5():
    rows = []
    with open(os.path.join(HERE, "golden", "tab5_porosity_permeability.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                e, k = line.split()
                rows.append((float(e), float(k)))
    return rows


def test_every_row_of_tab5_follows_the_fit():
    rows = tab5()
    assert len(rows) == 9
    for e, k in rows:
        assert permeability_from_porosity(e) == pytest.approx(k, rel=5e-3), e


def test_inverse_recovers_the_printed_porosities():
    for e, k in tab5():
        # the table prints K to three digits: the porosity is pinned to the
        # same relative precision through dK/K = (3/e + 2/(1-e)) de
        assert porosity_from_permeability(k) == pytest.approx(e, rel=2e-3), e


def test_round_trip_and_monotonicity():
    prev = -1.0
    for i in range(1, 99):
        e = i / 100.0
        k = permeability_from_porosity(e)
        assert k > prev
        prev = k
        assert porosity_from_permeability(k) == pytest.approx(e, rel=1e-12, abs=1e-15)


def test_limits():
    assert permeability_from_porosity(0.0) == 0.0
    assert porosity_from_permeability(0.0) == 0.0
    assert permeability_from_porosity(0.5) == pytest.approx(KOZENY_CARMAN_C * 0.5)
    with pytest.raises(ValueError):
        permeability_from_porosity(1.0)
    with pytest.raises(ValueError):
        permeability_from_porosity(-0.1)
    with pytest.raises(ValueError):
        porosity_from_permeability(-1.0)
