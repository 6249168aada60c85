"""Argument checks the C ABI makes before any device work (no GPU): bad
index parameters, bad mapping tables, bad network shapes and NULL handles
return SINN_EINVAL and hand out no object."""
import ctypes as C

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2301_10622_gb300 import sinnamon  # noqa: E402


@pytest.mark.parametrize("cfg", [
    dict(n=0, m=16, h=1), dict(n=100, m=0, h=1), dict(n=100, m=16, h=0),
    dict(n=100, m=4, h=5), dict(n=100, m=64, h=9), dict(n=100, m=4097, h=1),
    dict(n=100, m=16, h=1, tile_docs=512), dict(n=100, m=16, h=1, tile_docs=3000),
    dict(n=100, m=16, h=1, tile_docs=32768), dict(n=100, m=16, h=1, flags=4),
])
def test_bad_index_parameters(cfg):
    with pytest.raises(sinnamon.SinnError) as e:
        sinnamon.sinn_create_ex(**cfg)
    assert e.value.code == sinnamon.SINN_EINVAL


def test_bad_mapping_table():
    table = np.zeros(100, np.uint32)
    table[37] = 16  # outside [0, m)
    with pytest.raises(sinnamon.SinnError) as e:
        sinnamon.sinn_create_ex(100, 16, 1, table=table)
    assert e.value.code == sinnamon.SINN_EINVAL


@pytest.mark.parametrize("n_in,hidden", [(0, 64), (19, 0), (19, 4097), (1025, 64)])
def test_bad_network_shapes(n_in, hidden):
    lib = sinnamon.load()
    out = C.c_void_p(99)
    assert lib.sinn_mlp_create(n_in, hidden, 1, C.byref(out)) == sinnamon.SINN_EINVAL
    assert out.value is None


def test_null_handles():
    lib = sinnamon.load()
    assert lib.sinn_destroy(None) == sinnamon.SINN_OK
    assert lib.sinn_mlp_destroy(None) == sinnamon.SINN_OK
    calls = [("sinn_sync", (None, None)), ("sinn_insert", (None, None, None, None, 1, None, None)),
             ("sinn_delete", (None, None, 1, None)), ("sinn_mlp_sync", (None, None)),
             ("sinn_set_budget", (None, 5))]
    for name, args in calls:
        assert getattr(lib, name)(*args) == sinnamon.SINN_EINVAL, name
    assert lib.sinn_get_budget(None) == 0
    assert lib.sinn_create_ex(None, C.byref(C.c_void_p())) == sinnamon.SINN_EINVAL
