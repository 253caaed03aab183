"""__graft_entry__.smoke(): one small lambda-thinning run on cuda:0 through the
C-ABI, checked against the CPU oracle inside the function itself."""
import pytest

import __graft_entry__

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_smoke_runs_and_checks_itself():
    __graft_entry__.smoke()
