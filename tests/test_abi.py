"""The C-ABI library loads, exports every declared symbol, and its host-only
grid builder agrees with the oracle's independent construction (no GPU)."""
import os
import re

import numpy as np
import pytest

from paper_2406_18479_gb300 import gw
from oracle import grids

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-zA-Z0-9_]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert _declared() == sorted(gw.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol():
    L = gw.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert "sm_103a" in gw.gw_version()


@pytest.mark.parametrize("ntau,beta", [(1, 3.0), (2, 5.0), (7, 10.0), (32, 50.0), (100, 100.0), (120, 200.0)])
@pytest.mark.parametrize("stat", [0, 1])
def test_grid_builder_matches_oracle(ntau, beta, stat):
    tau, idx, F, B = gw.gw_grid_build(ntau, beta, stat)
    m, Fo, Bo = grids.transform_matrices(ntau, beta, stat)
    assert np.array_equal(idx, m)
    assert np.allclose(tau, grids.chebyshev_nodes(ntau, beta), rtol=0, atol=1e-13 * beta)
    assert np.abs(F - Fo).max() < 1e-13 * np.abs(Fo).max()
    assert np.abs(B - Bo).max() < 1e-11 * np.abs(Bo).max()
    assert np.abs(B @ F - np.eye(ntau)).max() < 1e-12


def test_sample_count_rule():
    for n in range(1, 40):
        assert gw.gw_sample_count(n, 0) % 2 == 1 and gw.gw_sample_count(n, 0) in (n, n + 1)
        assert gw.gw_sample_count(n, 1) % 2 == 0 and gw.gw_sample_count(n, 1) in (n, n + 1)
    assert gw.gw_sample_count(0, 0) == -1
    assert gw.gw_sample_count(4, 2) == -1
