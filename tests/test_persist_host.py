"""sinn_load's checks of a file before it touches the device (no GPU): a
missing, empty or foreign file, another format version, parameters that
sinn_create_ex would refuse, counters that do not fit the capacity, a
truncated mapping table and a table entry outside [0, m) are all refused
with SINN_EIO, and no index is returned."""
import ctypes as C
import struct

import pytest

pytest.importorskip("torch")

from paper_2301_10622_gb300 import sinnamon  # noqa: E402

# the file header: magic, version, n, m, h, T, flags, max_qnnz, sk_elem, then
# seed, cap, next_id, live_count, fwd_used, fwd_cap, budget, scratch_budget,
# tombstones, then the 8-field tuning
FMT = "<8s8I9Q8I"


def _header(**over):
    f = dict(magic=b"SINNIDX1", version=1, n=100, m=16, h=1, T=1024, flags=0, max_qnnz=64,
             sk_elem=4, seed=0x5151, cap=1024, next_id=10, live_count=8, fwd_used=80,
             fwd_cap=65536, budget=0, scratch_budget=1 << 30, tombstones=0)
    f.update(over)
    tune = (4, 32, 0, 0, 4, 4, 0, 0)
    return struct.pack(FMT, f["magic"], f["version"], f["n"], f["m"], f["h"], f["T"],
                       f["flags"], f["max_qnnz"], f["sk_elem"], f["seed"], f["cap"],
                       f["next_id"], f["live_count"], f["fwd_used"], f["fwd_cap"], f["budget"],
                       f["scratch_budget"], f["tombstones"], *tune)


def _table(n, h, m, bad=False):
    vals = [(j * 7 + o) % m for j in range(n) for o in range(h)]
    if bad:
        vals[5] = m
    return struct.pack("<Q", 4 * n * h) + struct.pack(f"<{n * h}I", *vals)


def _load(path):
    lib = sinnamon.load()
    out = C.c_void_p(1234)
    rc = lib.sinn_load(str(path).encode(), C.byref(out))
    return rc, out.value


def test_header_size():
    assert struct.calcsize(FMT) == 144


@pytest.mark.parametrize("name,content", [
    ("empty", b""),
    ("foreign", b"not a saved index" * 20),
    ("short header", _header()[:100]),
    ("version", _header(version=2) + _table(100, 1, 16)),
    ("m = 0", _header(m=0) + _table(100, 1, 16)),
    ("h > m", _header(h=20) + _table(100, 20, 16)),
    ("T not a power of two", _header(T=3000) + _table(100, 1, 16)),
    ("capacity not whole tiles", _header(cap=1500) + _table(100, 1, 16)),
    ("next id past capacity", _header(next_id=5000) + _table(100, 1, 16)),
    ("more live than ids", _header(live_count=11) + _table(100, 1, 16)),
    ("store over its size", _header(fwd_used=70000) + _table(100, 1, 16)),
    ("sketch element size", _header(sk_elem=2) + _table(100, 1, 16)),
    ("unknown flag", _header(flags=8) + _table(100, 1, 16)),
    ("truncated table", _header() + _table(100, 1, 16)[:200]),
    ("table length", _header() + struct.pack("<Q", 12) + b"\0" * 12),
    ("bin out of range", _header() + _table(100, 1, 16, bad=True)),
])
def test_bad_files_are_refused_before_the_device(tmp_path, name, content):
    p = tmp_path / "x.sinn"
    p.write_bytes(content)
    rc, out = _load(p)
    assert rc == sinnamon.SINN_EIO, name
    assert out is None


def test_missing_file(tmp_path):
    rc, out = _load(tmp_path / "none.sinn")
    assert rc == sinnamon.SINN_EIO and out is None
    lib = sinnamon.load()
    assert lib.sinn_save(None, b"x") == sinnamon.SINN_EINVAL
    assert lib.sinn_load(None, C.byref(C.c_void_p())) == sinnamon.SINN_EINVAL
