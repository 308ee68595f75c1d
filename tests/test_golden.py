"""The stored oracle fixtures (tests/golden) reproduce on this machine."""
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _lines():
    with open(os.path.join(HERE, "golden", "bernoulli64_dmax16.txt")) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("line", _lines())
def test_bernoulli64_fixture(line):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    seed = int(line.split()[0])
    assert mg.field_line(seed) == line
