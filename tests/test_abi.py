"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads
without a GPU, exports every symbol of include/mls6.h, and its host-only
logic (grid sizing, coarsest-level Ewald tables, argument validation)
agrees with the oracle, which computes the same quantities independently."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1308_4005_gb300 import build as B
from paper_1308_4005_gb300 import mls6

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mls6.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "mls6.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mls6_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree(lib):
    assert sorted(mls6.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_grid_dims_match_oracle(lib, orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        L = rng.uniform(3.0, 200.0, 3)
        h = rng.uniform(0.3, 3.0)
        lev = int(rng.integers(1, 6))
        assert mls6.mls6_grid_dims(L, h, lev) == orc.grid_dims(L, h, lev)


def test_grid_dims_refuse_grids_beyond_32_bit_node_indices(lib):
    """The grid kernels index nodes with 32-bit integers: a finest grid of
    more than 2^31 - 1 nodes is refused (MLS6_ERR_SIZE), one just below is
    accepted."""
    assert mls6.mls6_grid_dims((1290.0, 1290.0, 1290.0), 1.0, 1) == (1290, 1290, 1290)
    with pytest.raises(mls6.MLS6Error) as e:
        mls6.mls6_grid_dims((1291.0, 1291.0, 1291.0), 1.0, 1)
    assert e.value.code == mls6.MLS6_ERR_SIZE


@pytest.mark.parametrize("box,nl,l,a", [
    ((10.0, 10.0, 10.0), (3, 3, 3), 3, 2.5),
    ((40.0, 40.0, 120.0), (4, 4, 12), 4, 3.0),
    ((8.0, 9.0, 10.0), (3, 4, 5), 3, 1.0),
    ((6.0, 6.0, 6.0), (8, 8, 8), 1, 2.0),
])
def test_coarse_tables_ewald_vs_oracle_direct_sum(lib, orc, box, nl, l, a):
    """The library evaluates the coarsest-level lattice sums by Ewald
    summation; the oracle by direct image summation plus continuum tail.
    Two different methods for Eq. (last-grid-periodic-transformed)."""
    T, V = mls6.mls6_coarse_tables(box, nl, l, a)
    To, Vo = orc.top_table(box, a, nl, l)
    assert np.abs(T - To).max() <= 1e-13 * np.abs(To).max()
    assert np.abs(V - Vo).max() <= 5e-13 * np.abs(Vo).max()


def test_plan_argument_validation_needs_no_gpu(lib):
    h = C.c_void_p()
    box = mls6._darr((10.0, 10.0, 10.0))
    for order in (0, 2, 4, 6, 7):  # interpolation orders 3 and 5 only
        assert lib.mls6_plan(C.byref(h), box, 100, 2.5, 1.0, 3, order, 0) == mls6.MLS6_ERR_ORDER
    assert lib.mls6_plan(C.byref(h), box, -1, 2.5, 1.0, 3, 3, 0) == mls6.MLS6_ERR_ARG
    assert lib.mls6_plan(C.byref(h), box, 100, 0.0, 1.0, 3, 3, 0) == mls6.MLS6_ERR_ARG
    assert lib.mls6_plan(C.byref(h), box, 100, 2.5, -1.0, 3, 3, 0) == mls6.MLS6_ERR_ARG
    assert lib.mls6_plan(C.byref(h), box, 100, 2.5, 1.0, -1, 3, 0) == mls6.MLS6_ERR_GRID
    assert lib.mls6_plan(C.byref(h), box, 100, 2.5, 1.0, 3, 3, 7) == mls6.MLS6_ERR_ARG
    bad = mls6._darr((10.0, -1.0, 10.0))
    assert lib.mls6_plan(C.byref(h), bad, 100, 2.5, 1.0, 3, 3, 0) == mls6.MLS6_ERR_BOX
    assert lib.mls6_plan(None, box, 100, 2.5, 1.0, 3, 3, 0) == mls6.MLS6_ERR_ARG
    for n, st in ((5, 0), (-2, 0), (2, 3), (2, -1)):  # options out of range
        opt = mls6.PlanOptions(n, st)
        assert lib.mls6_plan_ex(C.byref(h), box, 100, 2.5, 1.0, 3, 3, 0, C.byref(opt)) == \
            mls6.MLS6_ERR_ARG
    assert mls6.status_string(mls6.MLS6_ERR_NONFINITE).startswith("non-finite")
    assert mls6.status_string(mls6.MLS6_ERR_TIMEOUT).startswith("a bounded")


def test_null_plan_calls_are_errors(lib):
    assert lib.mls6_eval(None, None, None, None, None, None) == mls6.MLS6_ERR_ARG
    assert lib.mls6_last_error(None) == mls6.MLS6_ERR_ARG
    lib.mls6_destroy(None)
