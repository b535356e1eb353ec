"""The C ABI on the CPU: the library builds for sm_103a, loads, and exports every symbol
that include/tucker.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "tucker.h")) as f:
        text = "\n".join(line for line in f if not line.lstrip().startswith("#"))
    return sorted(set(re.findall(r"TUCKER_API\s+[\w\s\*]*?\b(\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("tucker_init", "ttmc_mode", "qrp_leading", "hooi_iter", "core_tensor", "tucker_loss_grad",
                 "tucker_free"):
        assert name in syms


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2010_10638_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_2010_10638_gb300 import tucker
    for s in declared_symbols():
        assert hasattr(tucker, s), s
    assert sorted(tucker.EXPORTS) == sorted(declared_symbols())


def test_status_strings_without_a_gpu():
    from paper_2010_10638_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.tucker_status_str.restype = ctypes.c_char_p
    assert lib.tucker_status_str(0) == b"ok"
    assert lib.tucker_status_str(2) == b"rank out of range"


def test_normal_build_has_no_index_checks():
    """tucker_check_site is -1 in the normal build (no checks compiled in, no CUDA call)."""
    from paper_2010_10638_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.tucker_check_site.restype = ctypes.c_int32
    assert lib.tucker_check_site() == -1


def test_binding_flags_match_the_header():
    """Every TUCKER_F_* flag of the header has the same value in the binding, and no two
    flags share a bit."""
    with open(os.path.join(ROOT, "include", "tucker.h")) as f:
        text = f.read()
    from paper_2010_10638_gb300 import tucker
    flags = {k: int(v, 16) for k, v in re.findall(r"#define\s+(TUCKER_F_\w+)\s+(0x[0-9a-fA-F]+)u", text)}
    assert "TUCKER_F_TTMC_NORMS" in flags and len(flags) >= 6
    for name, value in flags.items():
        assert getattr(tucker, name) == value, name
    bits = list(flags.values())
    assert all(b & (b - 1) == 0 for b in bits) and len(set(bits)) == len(bits)


def test_device_entry_points_refuse_host_tensors():
    """No host fallback: the device entry points reject CPU tensors and other dtypes
    before any call into the library."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2010_10638_gb300 import build, tucker
    build.build()
    tucker.load()
    with pytest.raises(TypeError, match="CUDA tensor"):
        tucker.qrp_leading(torch.zeros(8, 4, dtype=torch.float64), 2)
    with pytest.raises(TypeError, match="CUDA tensor"):
        tucker.qrp_leading_noalloc(torch.zeros(8, 4, dtype=torch.float32), 2)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises instead of computing anything."""
    import pytest
    from paper_2010_10638_gb300 import tucker
    monkeypatch.setattr(tucker, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        tucker.load(str(tmp_path / "libtucker.so"))
