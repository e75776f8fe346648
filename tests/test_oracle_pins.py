"""The FP64 oracle against brute force, closed forms and invariants (CPU only)."""
import pytest

import pins
from oracle import galario_oracle as O


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    check(O)


def test_paper_templates_hankel():
    """Templates (a), (b), (d) of Sect. 5 against quadrature of the Hankel transform."""
    pytest.importorskip("scipy")
    pins.check_paper_templates_hankel(O)
