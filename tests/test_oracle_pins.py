"""The oracle against facts fixed by the paper and by mathematics (CPU only)."""
import pytest

import oracle_pins as P  # noqa: E402


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


def test_tables_1_2_iteration_counts():
    # Tables 1 and 2: mean RGDBEK and GDBEK iterations on 99%-sparse random
    # matrices, within 20% of the printed values.
    P.pin_tables_1_2()
