"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol that
include/addker.h declares, and rejects bad arguments on the host (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "addker.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_17344_gb300 import native
    return native.lib()


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(addker_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("addker_setup", "addker_matvec", "addker_dmatvec", "addker_matvec_all", "addker_free",
                     "addker_strerror", "addker_prescale", "addker_set_params"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_rate_library_is_apart_from_the_product(lib):
    """The device-rate microbenchmark (include/addker_rates.h) is measurement tooling: its own library
    exports it and the product library does not."""
    from paper_2404_17344_gb300 import rates
    names = declared_functions(os.path.join(ROOT, "include", "addker_rates.h"))
    assert names == ["addker_device_rates"]
    rl = rates.lib()
    for name in names:
        assert hasattr(rl, name), name
        assert not hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2404_17344_gb300 import native
    assert sorted(native.SIGNATURES) == declared_functions()


def test_status_codes_match_header():
    from paper_2404_17344_gb300 import native
    text = open(HEADER).read()
    for name in ("ADDKER_OK", "ADDKER_EINVAL", "ADDKER_EDOMAIN", "ADDKER_ENOMEM", "ADDKER_ECUDA",
                 "ADDKER_ETIMEOUT", "ADDKER_ELIMIT", "ADDKER_ELL_SHARED", "ADDKER_SIGMA_F", "ADDKER_WIN_KB",
                 "ADDKER_WIN_ES", "ADDKER_KERNEL_GAUSS", "ADDKER_KERNEL_MATERN12", "ADDKER_REG_DEFAULT",
                 "ADDKER_REG_SEPARABLE", "ADDKER_REG_RADIAL"):
        m = re.search(rf"#define {name}\s+\(?(-?\d+)\)?", text)
        assert m and int(m.group(1)) == getattr(native, name), name


def test_strerror_and_defaults(lib):
    from paper_2404_17344_gb300 import native
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(lib.addker_strerror(code), bytes)
    o = native.addker_opts()
    assert lib.addker_opts_default(ctypes.byref(o)) == 0
    assert o.sigma_os == 2.0 and o.eps_B == 1 / 16 and o.p == -1 and o.kernel == native.ADDKER_KERNEL_GAUSS
    assert o.window == native.ADDKER_WIN_KB
    assert o.compensated == 0 and o.reg == native.ADDKER_REG_DEFAULT and ctypes.sizeof(o) == 48
    assert lib.addker_opts_default(None) == native.ADDKER_EINVAL
    assert lib.addker_free(None) == 0


def _setup(lib, **kw):
    from paper_2404_17344_gb300 import native
    args = dict(N=10, d=3, off=[0, 3], feat=[0, 1, 2], P=1, ell=[0.5], sigma_f=1.0, bw=[32], m=4)
    args.update(kw)
    plan = ctypes.c_void_p()
    off = (ctypes.c_int * len(args["off"]))(*args["off"])
    feat = (ctypes.c_int * max(1, len(args["feat"])))(*args["feat"])
    ell = (ctypes.c_double * max(1, len(args["ell"])))(*args["ell"])
    bw = (ctypes.c_int * max(1, len(args["bw"])))(*args["bw"])
    dummy = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first, or the pointer check rejects it
    return lib.addker_setup(ctypes.byref(plan), dummy, args["N"], args["d"], off, feat, args["P"], ell,
                            args["sigma_f"], bw, args["m"], None), plan


@pytest.mark.parametrize("kw", [
    dict(N=0), dict(d=0), dict(P=0), dict(bw=[31]), dict(bw=[2]), dict(bw=[66]), dict(m=1), dict(m=9),
    dict(ell=[0.0]), dict(ell=[-1.0]), dict(sigma_f=0.0), dict(off=[0, 4], feat=[0, 1, 2, 0]),
    dict(feat=[0, 1, 5]), dict(feat=[0, 1, 1]), dict(off=[1, 3]), dict(bw=[8], m=4),
])
def test_setup_rejects_bad_arguments(lib, kw):
    from paper_2404_17344_gb300 import native
    status, plan = _setup(lib, **kw)
    assert status == native.ADDKER_EINVAL
    assert not plan.value


def test_setup_rejects_host_pointer(lib):
    """A valid layout with a pointer that is not device memory is refused before any work."""
    from paper_2404_17344_gb300 import native
    status, plan = _setup(lib)
    assert status == native.ADDKER_EINVAL


def test_product_calls_reject_null_plan(lib):
    from paper_2404_17344_gb300 import native
    v = ctypes.c_void_p(0x1000)
    assert lib.addker_matvec(None, v, v, 1) == native.ADDKER_EINVAL
    assert lib.addker_matvec_all(None, v, v, v, 1) == native.ADDKER_EINVAL
    assert lib.addker_dmatvec(None, 0, v, v, 1) == native.ADDKER_EINVAL
    assert lib.addker_matvec_all_host(None, v, v, v, 1) == native.ADDKER_EINVAL
    assert lib.addker_set_params(None, None, 1.0) == native.ADDKER_EINVAL
    assert lib.addker_sync(None) == native.ADDKER_EINVAL
    assert lib.addker_set_precond(None, 1) == native.ADDKER_EINVAL
    assert lib.addker_set_schedule(None, 256, 256, 0, 0) == native.ADDKER_EINVAL


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and the binding raises if the library is missing."""
    pkg = os.path.join(ROOT, "paper_2404_17344_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "oracle" not in src.replace("the oracle", ""), f
            assert "workloads" not in src, f


def test_setup_rejects_unknown_kernel_family(lib):
    from paper_2404_17344_gb300 import native
    o = native.addker_opts()
    lib.addker_opts_default(ctypes.byref(o))
    o.kernel = 7
    plan = ctypes.c_void_p()
    off = (ctypes.c_int * 2)(0, 3)
    feat = (ctypes.c_int * 3)(0, 1, 2)
    ell = (ctypes.c_double * 1)(0.5)
    bw = (ctypes.c_int * 1)(32)
    st = lib.addker_setup(ctypes.byref(plan), ctypes.c_void_p(0x1000), 10, 3, off, feat, 1, ell, 1.0, bw, 4,
                          ctypes.byref(o))
    assert st == native.ADDKER_EINVAL and not plan.value


def test_setup_rejects_unknown_window(lib):
    from paper_2404_17344_gb300 import native
    o = native.addker_opts()
    lib.addker_opts_default(ctypes.byref(o))
    o.window = 2
    plan = ctypes.c_void_p()
    off = (ctypes.c_int * 2)(0, 3)
    feat = (ctypes.c_int * 3)(0, 1, 2)
    ell = (ctypes.c_double * 1)(0.5)
    bw = (ctypes.c_int * 1)(32)
    st = lib.addker_setup(ctypes.byref(plan), ctypes.c_void_p(0x1000), 10, 3, off, feat, 1, ell, 1.0, bw, 4,
                          ctypes.byref(o))
    assert st == native.ADDKER_EINVAL and not plan.value


@pytest.mark.parametrize("kernel,reg", [(0, 2), (0, -2), (1, 0)])
def test_setup_rejects_bad_regularisation_reading(lib, kernel, reg):
    """An unknown reading, or the separable reading with Matern(1/2) (whose kernel does not separate),
    is refused on the host."""
    from paper_2404_17344_gb300 import native
    o = native.addker_opts()
    lib.addker_opts_default(ctypes.byref(o))
    o.kernel, o.reg = kernel, reg
    plan = ctypes.c_void_p()
    off = (ctypes.c_int * 2)(0, 3)
    feat = (ctypes.c_int * 3)(0, 1, 2)
    ell = (ctypes.c_double * 1)(0.5)
    bw = (ctypes.c_int * 1)(32)
    st = lib.addker_setup(ctypes.byref(plan), ctypes.c_void_p(0x1000), 10, 3, off, feat, 1, ell, 1.0, bw, 4,
                          ctypes.byref(o))
    assert st == native.ADDKER_EINVAL and not plan.value
