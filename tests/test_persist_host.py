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


# ---- payload checks: a whole small index written in the file format, then
# one entry of what the kernels index through damaged at a time

def _index_file(corrupt=None):
    """A saved index of n=100, m=16, h=1, T=1024 (one tile): ids 0..9 handed
    out, 3 and 7 deleted (free), the others live with 10 entries each; one
    array container per coordinate.  `corrupt` names one damage to apply."""
    import numpy as np
    n, m, T, cap = 100, 16, 1024, 1024
    rng = np.random.default_rng(5)
    ids = np.arange(10)
    free = [3, 7]
    live = np.zeros(cap, np.uint8)
    live[[i for i in ids if i not in free]] = 1
    vecs = [np.sort(rng.choice(n, 10, replace=False)).astype(np.uint32) for _ in ids]
    fwd = np.zeros((100, 2), np.uint32)
    fwd_off = np.zeros(cap, np.uint64)
    fwd_nnz = np.zeros(cap, np.uint32)
    nnz = np.zeros(cap, np.uint32)
    for i in ids:
        fwd[10 * i:10 * i + 10, 0] = vecs[i]
        fwd[10 * i:10 * i + 10, 1] = np.float32(1.5).view(np.uint32)
        fwd_off[i], fwd_nnz[i] = 10 * i, 10
        if live[i]:
            nnz[i] = 10
    # the tile's containers: per coordinate, the sorted live ids holding it
    posts = {j: [i for i in ids if live[i] and j in vecs[i]] for j in range(n)}
    dirs = np.zeros((n, 2), np.uint32)
    words, run = [], 0
    for j in range(n):
        if posts[j]:
            dirs[j] = (run, len(posts[j]))
            words += posts[j]
            run += len(posts[j])
    post_cap = 128
    words = np.array(words + [0] * (post_cap - len(words)), np.uint16)
    coord_len = np.array([len(posts[j]) for j in range(n)], np.uint32)
    live_bits = np.zeros(cap // 32, np.uint32)
    for i in np.nonzero(live)[0]:
        live_bits[i >> 5] |= np.uint32(1 << (i & 31))
    tile_nnz = np.array([int(nnz.sum())], np.uint64)
    post_len = np.array([run], np.uint64)
    free_arr = np.array(free, np.uint32)
    hdr = dict(n=n, m=m, h=1, T=T, cap=cap, next_id=10, live_count=int(live.sum()),
               fwd_used=100, fwd_cap=65536)
    if corrupt == "live bit":
        live_bits[0] ^= np.uint32(1 << 3)           # a free id's device bit set
    elif corrupt == "store offset":
        fwd_off[0] = 95                              # 95 + 10 > 100 entries used
    elif corrupt == "store count":
        fwd_nnz[1] = 9                               # differs from the host count
    elif corrupt == "store coordinate":
        fwd[12, 0] = n                               # a coordinate outside [0, n)
    elif corrupt == "container past storage":
        j = int(np.nonzero(dirs[:, 1])[0][0])
        dirs[j, 0] = post_cap - int(dirs[j, 1]) + 1  # its last entry is past the words
    elif corrupt == "local id":
        words[0] = T + 1                             # an array entry outside the tile
    elif corrupt == "bitmap alignment":
        j = int(np.nonzero(dirs[:, 1] == 0)[0][0])
        dirs[j] = (1, T // 8)                        # a bitmap at an odd word
    elif corrupt == "tile entries":
        tile_nnz[0] += 1
    elif corrupt == "free id live":
        free_arr[0] = 4
    elif corrupt == "free id repeated":
        free_arr[1] = 3
    elif corrupt == "storage without containers":
        post_cap = 0
    table = [(j * 7) % m for j in range(n)]

    def arr(a):
        b = np.ascontiguousarray(a).tobytes()
        return struct.pack("<Q", len(b)) + b

    plane = np.zeros(m * cap, np.float32)
    out = _header(**hdr) + struct.pack("<Q", 4 * n) + struct.pack(f"<{n}I", *table)
    out += arr(plane) + arr(plane) + arr(live_bits) + arr(fwd_off) + arr(fwd_nnz) + arr(fwd)
    out += arr(dirs) + arr(coord_len) + arr(live) + arr(nnz) + arr(free_arr)
    out += arr(post_len) + arr(np.array([post_cap], np.uint64)) + arr(tile_nnz)
    out += arr(np.zeros(1, np.uint64))
    out += arr(words[:post_cap])
    return out


def test_a_sound_index_file_passes_the_checks(tmp_path):
    """The undamaged file gets past every check: without a GPU the load then
    fails creating the index on the device (never SINN_EIO)."""
    p = tmp_path / "ok.sinn"
    p.write_bytes(_index_file())
    rc, out = _load(p)
    if rc == sinnamon.SINN_OK:      # run where a GPU is present
        assert sinnamon.load().sinn_destroy(C.c_void_p(out)) == sinnamon.SINN_OK
        return
    assert rc in (sinnamon.SINN_ECUDA, sinnamon.SINN_ENOMEM), rc
    assert out is None


@pytest.mark.parametrize("damage", [
    "live bit", "store offset", "store count", "store coordinate", "container past storage",
    "local id", "bitmap alignment", "tile entries", "free id live", "free id repeated",
    "storage without containers"])
def test_damaged_payload_is_refused_before_the_device(tmp_path, damage):
    p = tmp_path / "bad.sinn"
    p.write_bytes(_index_file(damage))
    rc, out = _load(p)
    assert rc == sinnamon.SINN_EIO, damage
    assert out is None


def test_truncated_payload_is_refused(tmp_path):
    full = _index_file()
    for cut in (len(full) - 1, len(full) - 300, len(full) // 2):
        p = tmp_path / f"cut{cut}.sinn"
        p.write_bytes(full[:cut])
        rc, out = _load(p)
        assert rc == sinnamon.SINN_EIO and out is None
