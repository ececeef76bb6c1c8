"""CPU-only checks of the CUDA library: it builds, loads, exports every entry
point that include/dg.h declares, and its host-side basis agrees with the
closed forms (no kernel is launched here)."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import dg


def test_library_exports_every_header_symbol():
    L = dg.lib()
    names = dg.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_host_lgl_nodes(ora, N):
    x, w = dg.lgl_nodes(N)
    xo, wo, Do = ora.lgl(N)
    assert np.abs(x - xo).max() < 4e-16 * N
    assert np.abs(w - wo).max() < 1e-15 * N
    if N == 3:
        assert np.allclose(x, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], rtol=0, atol=1e-16)


def test_host_lgl_rejects_bad_degree():
    with pytest.raises(dg.DGError) as e:
        dg.lgl_nodes(0)
    assert e.value.code == -1


def test_bounds_checking_build_exports_every_header_symbol():
    """The bounds-checking variant (DG_DEBUG_BOUNDS) builds and exports the
    same C ABI."""
    import ctypes
    from paper_2606_18927_gb300 import build
    L = ctypes.CDLL(build.build(variant="debug"))
    missing = [n for n in dg.header_functions() if not hasattr(L, n)]
    assert not missing, missing
