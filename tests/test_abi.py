"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every
entry point include/ept.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ept.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ept_[a-z_0-9]+)\s*\(", text)))


def _device_present():
    torch = pytest.importorskip("torch")
    return torch.cuda.is_available()


@pytest.fixture(scope="module")
def lib_path():
    from paper_2406_06488_gb300 import _build
    return _build.build()


def test_header_and_binding_agree():
    from paper_2406_06488_gb300 import ept
    assert _declared() == sorted(ept.EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_abi_version_and_errors_without_gpu(lib_path):
    from paper_2406_06488_gb300 import ept
    lib = ept.load()
    import re
    hdr = open(os.path.join(ROOT, "include", "ept.h")).read()
    want = int(re.search(r"#define EPT_ABI_VERSION (\d+)", hdr).group(1))
    from paper_2406_06488_gb300 import ept
    assert lib.ept_abi_version() == want == ept.ABI_VERSION
    # creating a context without a GPU fails cleanly with a status, not a crash (with
    # one, it succeeds)
    h = ctypes.c_void_p()
    st = lib.ept_create(ctypes.byref(h), 0, 0)
    if _device_present():
        assert st == 0
        lib.ept_destroy(h)
    else:
        assert st != 0
        assert isinstance(lib.ept_last_error(), bytes)
    # size estimates are pure host arithmetic
    assert ept.estimate_bytes(2000, 3000, 1000, 10000) > 0
    assert ept.estimate_bytes(0, 3, 1, 1) == 0
    assert ept.estimate_bytes(2, 3, (1 << 30) + 1, 1) == 0       # p beyond 2^30
    assert ept.estimate_bytes(2, 3, 1 << 30, 1) > 0
    assert ept.estimate_bytes(1 << 21, (1 << 21) + 1, 1, 1) == 0  # nx + ny beyond 2^22


def test_option_tables_agree():
    # the header's option numbers, the binding's option names and the environment
    # variables that give their starting values (every option but the test hooks)
    from paper_2406_06488_gb300 import ept
    hdr = open(os.path.join(ROOT, "include", "ept.h")).read()
    declared = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"EPT_OPT_([A-Z_]+) = (\d+)", hdr)}
    assert declared == ept.OPTION
    src = open(os.path.join(ROOT, "paper_2406_06488_gb300", "csrc", "ept_api.cu")).read()
    env = dict(re.findall(r'\{"EPT_([A-Z_]+)", EPT_OPT_([A-Z_]+)\}', src))
    assert all(k == v for k, v in env.items())
    hooks = {"fault_inject_alloc", "fault_inject_stall"}
    assert {k.lower() for k in env} == set(declared) - hooks
    for k in env:   # and the header's list of environment variables names each one
        assert "EPT_" + k in hdr


def test_build_info_names_this_machine(lib_path):
    # the library is compiled where it runs: its host architecture is this machine's
    import platform
    from paper_2406_06488_gb300 import ept
    info = ept.build_info()
    assert "host %s;" % platform.machine() in info, info
    assert "device sm_103a;" in info and "abi %d;" % ept.ABI_VERSION in info, info


def test_destroy_null_is_ok(lib_path):
    from paper_2406_06488_gb300 import ept
    assert ept.load().ept_destroy(None) == 0


def test_host_side_argument_checks(lib_path):
    # checks that run before any device call, so they hold on a machine without a GPU
    from paper_2406_06488_gb300 import ept
    lib = ept.load()
    h = ctypes.c_void_p()
    half = ept._Allocator(ept._ALLOC_FN(lambda n, s, u: None), ept._FREE_FN(), None)
    assert lib.ept_create_ex(ctypes.byref(h), 0, 0, ctypes.byref(half)) == 1   # alloc without free: EPT_EINVAL
    assert b"alloc and free" in lib.ept_last_error()
    assert lib.ept_create_ex(None, 0, 0, None) == 1
    assert lib.ept_set_option(None, 9, 1) == 1
    r = ept._Result()
    assert lib.ept_test(None, None, 1, None, 1, 1, 0, 0, 1.0, 1, ctypes.c_uint64(0), 1, None, ctypes.byref(r),
                        None) == 1
    # the pre-computation baseline: estimate = the full n x n matrix and the rest
    n = 3000
    est = ept.estimate_bytes(1500, 1500, 64, 200, prec="pooled_fp32")
    assert est >= ((n + 255) // 256 * 256) ** 2 * 4
    assert ept.estimate_bytes(1500, 1500, 64, 200, prec=7) == 0


def test_environment_options_are_checked(lib_path, monkeypatch):
    # EPT_<OPTION> values are parsed at ept_create; without a GPU the call fails earlier
    # (no device), so there only the library's acceptance of the names is exercised;
    # with one, a valid value gives a context
    from paper_2406_06488_gb300 import ept
    monkeypatch.setenv("EPT_WAIT_LIMIT_MS", "250")
    h = ctypes.c_void_p()
    st = ept.load().ept_create(ctypes.byref(h), 0, 0)
    if _device_present():
        assert st == 0
        ept.load().ept_destroy(h)
    else:
        assert st != 0
