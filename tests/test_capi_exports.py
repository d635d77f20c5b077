"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares (no compute calls here)."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def declared_functions() -> set[str]:
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)          # drop comments
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in {"if", "while", "for", "return", "sizeof"}:
                names.add(name)
    return names


@pytest.fixture(scope="module")
def so_path():
    import __graft_entry__
    from paper_2602_04103_gb300 import _build
    _build.build_cuda()
    return _build.QR_SO


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["qr_build", "qr_rank", "qr_rank4", "qr_rank_c", "qr_free", "qr_status", "qr_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(so_path):
    lib = ctypes.CDLL(str(so_path))
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, f"declared in include/*.h but not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", str(so_path)], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared_functions() <= exported


def test_binding_loads_and_reports_errors_without_gpu(so_path):
    from paper_2602_04103_gb300 import capi
    assert capi.lib.qr_abi_version() == 1
    # argument errors are caught on the host before any CUDA call
    h = ctypes.c_void_p()
    assert capi.lib.qr_build(None, 10, 3, 0, None, ctypes.byref(h)) == capi.QR_EINVAL
    assert b"sigma" in capi.lib.qr_last_error()
    assert capi.lib.qr_build(None, 1 << 43, 2, 0, None, ctypes.byref(h)) == capi.QR_EINVAL
    assert capi.lib.qr_rank(None, None, 0, 1, None, None) == capi.QR_EINVAL


def test_binding_constants_match_the_headers():
    """Every QR_* / QFM_* constant the binding names has the header's value."""
    from paper_2602_04103_gb300 import capi
    defines = {}
    for h in (ROOT / "include").glob("*.h"):
        for m in re.finditer(r"^#define\s+((?:QR|QFM)_\w+)\s+\(?(-?\d+)", h.read_text(), flags=re.M):
            defines[m.group(1)] = int(m.group(2))
    named = [k for k in dir(capi) if re.fullmatch(r"(QR|QFM)_[A-Z0-9_]+", k)]
    assert "QR_LAYOUT_INLINE24_8" in named
    for k in named:
        assert k in defines and defines[k] == getattr(capi, k), k


def test_layout_rules_checked_on_the_host(so_path):
    """qr_build_ex refuses a layout the alphabet does not have before any CUDA
    call: BiRank32x2 is sigma 2 only, QuadRank24_8 sigma 4 only."""
    from paper_2602_04103_gb300 import capi
    h = ctypes.c_void_p()
    word = (ctypes.c_uint64 * 1)(0)
    for sigma, layout in ((4, capi.QR_LAYOUT_INLINE32X2), (2, capi.QR_LAYOUT_INLINE24_8), (2, 6), (4, -1)):
        rc = capi.lib.qr_build_ex(word, 10, sigma, 0, layout, None, ctypes.byref(h))
        assert rc == capi.QR_EINVAL and not h.value, (sigma, layout)
    capi.lib.qr_build_ex(word, 10, 2, 0, capi.QR_LAYOUT_INLINE24_8, None, ctypes.byref(h))
    assert b"sigma 4 only" in capi.lib.qr_last_error()


def test_division_constants():
    # floor(q / 496) and floor(q / 224) by multiply-high, as the kernels compute them
    import random
    M31, M7 = 0x8421084210842109, 0x924924924924924A
    rnd = random.Random(1)
    qs = [0, 1, 495, 496, 497, 223, 224, 225, (1 << 43) - 1, (1 << 45) - 1, (1 << 63) - 1]
    qs += [rnd.getrandbits(63) for _ in range(20000)] + [rnd.randrange(0, 1 << 20) for _ in range(20000)]
    for q in qs:
        assert ((q >> 4) * M31 >> 64) >> 4 == q // 496
        assert ((q >> 5) * M7 >> 64) >> 2 == q // 224
    src = (ROOT / "paper_2602_04103_gb300" / "csrc" / "qr_common.cuh").read_text()
    assert "0x8421084210842109" in src and "0x924924924924924A" in src


def test_division_constants_sector_and_32bit():
    """The other line-index divisions: 480 = 32 * 15 and 192 = 64 * 3 (sector
    layouts), 1008 = 16 * 63, and the 32-bit forms the region pass takes when
    n < 2^37 (q >> 5 or q >> 6 below 2^32).  Each 32-bit magic M = ceil(2^s / d)
    is exact for every x below 2^32 when (d M - 2^s) (2^32 - 1) < 2^s, the
    Granlund-Montgomery bound; the samples check it at the edges."""
    import random
    M15, M3, M63 = 0x8888888888888889, 0xAAAAAAAAAAAAAAAB, 0x8208208208208209
    m15, m3, m7 = 0x88888889, 0xAAAAAAAB, 0x24924925
    assert (15 * m15 - (1 << 35)) * ((1 << 32) - 1) < (1 << 35)
    assert (3 * m3 - (1 << 33)) * ((1 << 32) - 1) < (1 << 33)
    assert (7 * m7 - (1 << 32)) * ((1 << 27) - 1) < (1 << 32)   # div224_32: x < 2^27
    rnd = random.Random(2)
    edges = [0, 1, 191, 192, 193, 479, 480, 481, 1007, 1008, 1009, (1 << 37) - 1, (1 << 37) - 480, (1 << 36) + 7]
    qs = edges + [rnd.getrandbits(63) for _ in range(20000)] + [rnd.getrandbits(37) for _ in range(20000)]
    for q in qs:
        assert ((q >> 5) * M15 >> 64) >> 3 == q // 480
        assert ((q >> 6) * M3 >> 64) >> 1 == q // 192
        assert ((q >> 4) * M63 >> 64) >> 5 == q // 1008
        if q < (1 << 37):
            assert ((q >> 5) * m15 >> 32) >> 3 == q // 480
            assert ((q >> 6) * m3 >> 32) >> 1 == q // 192
        if q < (1 << 32):
            assert (q >> 5) * m7 >> 32 == q // 224
    # 448 = 64 * 7 (the 32-bit inline layout BiRank32x2): the 64-bit form with the magic of
    # div224, and the 32-bit form for q < 2^37 with M = ceil(2^34 / 7), exact for x < 2^32
    # while x (7 M - 2^34) < 2^34
    m7_34, M7 = 0x92492493, 0x924924924924924A
    assert m7_34 == -(-(1 << 34) // 7) and (7 * m7_34 - (1 << 34)) * ((1 << 32) - 1) < (1 << 34) * 7
    for q in qs + [(1 << 37) - 1, (1 << 37) - 448, 447, 448, 449]:
        assert ((q >> 6) * M7 >> 64) >> 2 == q // 448
        if q < (1 << 37):
            assert ((q >> 6) * m7_34 >> 32) >> 2 == q // 448
    for r in range(7):
        x = (1 << 31) - 1 - r
        assert (x * m7_34 >> 32) >> 2 == x // 7
    for d, M in ((15, m15), (3, m3)):   # the largest dividend below 2^32 of each residue
        for r in range(d):
            x = (1 << 32) - 1 - r
            assert (x * M >> 32) >> (3 if d == 15 else 1) == x // d
    src = (ROOT / "paper_2602_04103_gb300" / "csrc" / "qr_common.cuh").read_text()
    assert all(h in src for h in ("0x8888888888888889", "0xAAAAAAAAAAAAAAAB", "0x8208208208208209", "0x24924925"))
    reg = (ROOT / "paper_2602_04103_gb300" / "csrc" / "qr_region.cu").read_text()
    assert "0x88888889u" in reg and "0xAAAAAAABu" in reg and "0x92492493u" in reg


def test_handle_classes():
    # the FM handle offers count, not the rank calls of a rank index
    from paper_2602_04103_gb300 import capi
    assert not issubclass(capi.QFMIndex, capi.QRIndex)
    for name in ("rank", "rank4", "prefix_rank", "status", "free"):
        assert callable(getattr(capi.QRIndex, name))
    for name in ("count", "status", "free"):
        assert callable(getattr(capi.QFMIndex, name))
    assert not hasattr(capi.QFMIndex, "rank")
    idx = capi.QRIndex(None)       # an empty handle frees as a no-op
    idx.free()
