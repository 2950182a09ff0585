"""Plan files without a GPU (host-only plans): save -> load gives back every array bit for bit; a file that
is missing, truncated, of another format, fails its checksum or breaks a structural invariant is refused
with EHYB_ERR_IO before anything could be uploaded."""
import struct

import numpy as np
import pytest

import gen

HEADER = struct.Struct("<8sII4q8i18qQ")   # magic, version, header bytes, n/nnz/er_nnz/ell_nnz, 8 ints, 18 lengths, checksum
ARRAYS = [("new_to_old", 4), ("part_ptr", 4), ("slice_ptr", 4), ("slice_pos", 8), ("slice_order", 4), ("ell_col", 2),
          ("ell_val", 8), ("row_ell_count", 4), ("er_part_ptr", 4), ("er_row", 4), ("er_ptr", 8), ("er_col", 4),
          ("er_val", 8), ("er_slice_pos", 8), ("er_scol", 4), ("er_scol_old", 4), ("er_sval", 8), ("row_er_count", 4)]
KEYS = ("new_to_old", "part_ptr", "slice_ptr", "slice_pos", "ell_col", "ell_val", "row_ell_count", "er_part_ptr",
        "er_row", "er_ptr", "er_col", "er_val", "er_slice_pos", "er_scol", "er_sval", "row_er_count")


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    return m


def _fnv_words(payload: bytes) -> int:
    """FNV-1a over 64-bit little-endian words, the last one zero-padded (the file format's checksum)."""
    h = 1469598103934665603
    if len(payload) % 8:
        payload += b"\0" * (8 - len(payload) % 8)
    for (w,) in struct.iter_unpack("<Q", payload):
        h = ((h ^ w) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _offsets(blob: bytes):
    hdr = HEADER.unpack_from(blob)
    lens = hdr[15:33]
    off, out = HEADER.size, {}
    for (name, size), ln in zip(ARRAYS, lens):
        out[name] = (off, ln, size)
        off += ln * size
    return hdr, out


def _resign(blob: bytearray):
    hdr = list(HEADER.unpack_from(bytes(blob)))
    hdr[-1] = _fnv_words(bytes(blob[HEADER.size:]))
    HEADER.pack_into(blob, 0, *hdr)


OPTS = [dict(), dict(er_layout=1), dict(ell_tpr=2, slice_rows=300), dict(ell_width_cap=5, slice_rows=97)]


@pytest.mark.parametrize("opt", OPTS)
def test_round_trip_bit_identical(eh, tmp_path, opt):
    A = gen.random_csr(2500, 4, mean_row=9, empty_frac=0.05, long_rows=3, long_len=700, duplicates=True)
    P = eh.Plan(A, host_only=1, keep_host=1, **opt)
    f = str(tmp_path / "p.ehyb")
    P.save(f)
    Q = eh.Plan.load(f, host_only=1, keep_host=1)
    a, b = P.export(), Q.export()
    for k in KEYS + ("er_layout", "tpr", "nparts"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    ia, ib = P.info(), Q.info()
    for k in ("n", "nnz", "nparts", "ell_nnz", "er_nnz", "slice_rows", "ell_width_cap"):
        assert ia[k] == ib[k], k
    # the checksum the library wrote is the format's documented one
    blob = open(f, "rb").read()
    assert HEADER.unpack_from(blob)[-1] == _fnv_words(blob[HEADER.size:])


def test_bad_files_are_refused(eh, tmp_path):
    A = gen.fem2d_p1(N=30)
    P = eh.Plan(A, host_only=1, keep_host=1, slice_rows=100)
    f = tmp_path / "p.ehyb"
    P.save(str(f))
    good = f.read_bytes()

    def refused(blob, status=eh.EHYB_ERR_IO):
        g = tmp_path / "bad.ehyb"
        g.write_bytes(bytes(blob))
        with pytest.raises(eh.EhybError) as e:
            eh.Plan.load(str(g), host_only=1)
        assert e.value.status == status

    with pytest.raises(eh.EhybError) as e:
        eh.Plan.load(str(tmp_path / "missing.ehyb"), host_only=1)
    assert e.value.status == eh.EHYB_ERR_IO
    refused(good[:len(good) // 2])                       # truncated
    refused(b"XXXXXXXX" + good[8:])                      # another format
    bad = bytearray(good)
    bad[-3] ^= 0x40                                      # one flipped bit in the payload
    refused(bad)
    hdr, off = _offsets(good)
    # checksum-valid files that break an invariant the kernels index by
    o, ln, _ = off["new_to_old"]
    bad = bytearray(good)
    bad[o:o + 4] = bad[o + 4:o + 8]                      # not a permutation
    _resign(bad)
    refused(bad)
    o, ln, _ = off["ell_col"]
    bad = bytearray(good)
    struct.pack_into("<H", bad, o, 60000)                # a local column outside its partition
    _resign(bad)
    refused(bad)
    o, ln, _ = off["er_scol"]
    bad = bytearray(good)
    struct.pack_into("<i", bad, o, A.n)                  # a global column outside [0, n)
    _resign(bad)
    refused(bad)
    o, ln, _ = off["slice_order"]
    bad = bytearray(good)
    struct.pack_into("<i", bad, o, 10 ** 6)              # a slice id outside its partition
    _resign(bad)
    refused(bad)
    bad = bytearray(good)                                # the unchanged payload re-signed still loads
    _resign(bad)
    g = tmp_path / "ok.ehyb"
    g.write_bytes(bytes(bad))
    assert eh.Plan.load(str(g), host_only=1).info()["n"] == A.n
    with pytest.raises(eh.EhybError) as e:
        eh.Plan.load(str(f), host_only=1, lowp=3)
    assert e.value.status == 1
