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
