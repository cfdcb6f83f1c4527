"""CPU-side checks of the CUDA library: it loads, exports every entry point
its header declares, and its host-side geometry logic agrees with the
oracle's (two independent implementations of the same readings).  No
compute call is made here: that needs a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import build
    build.build()
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


def test_library_exports_every_header_symbol(fg):
    syms = fg.header_symbols()
    assert len(syms) >= 19
    lib = ctypes.CDLL(fg.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", fg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fl_\w+)", out))
    assert set(syms) <= exported


def test_peak_measurement_library_exports_its_header_symbols():
    """The roofline-ceiling library bench.py loads (libflpeaks) exports every
    function include/flpeaks.h declares; it is separate from libflashgpu."""
    from paper_2401_16732_gb300 import build
    path = build.build_peaks()
    with open(os.path.join(ROOT, "include", "flpeaks.h")) as f:
        syms = re.findall(r"^int (fl_\w+)\(", f.read(), re.M)
    assert syms == ["fl_measure_butterfly_rate", "fl_measure_tc_f16_rate"]
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(syms) <= set(re.findall(r" T (fl_\w+)", out))


GEOMS = [
    (4096, 16, 16, 16, 16, 3, 1, 1), (8192, 3, 64, 32, 32, 3, 1, 1), (8192, 64, 128, 32, 32, 3, 2, 1),
    (8192, 64, 128, 32, 32, 1, 2, 0), (8192, 512, 512, 4, 4, 3, 1, 1), (16384, 3, 64, 224, 224, 7, 2, 3),
    (16384, 256, 64, 56, 56, 1, 1, 0), (16384, 512, 2048, 7, 7, 1, 1, 0), (2048, 3, 4, 40, 40, 7, 2, 3),
    (64, 2, 3, 10, 10, 3, 1, 1), (256, 9, 2, 8, 8, 1, 2, 0), (2048, 5, 5, 31, 17, 5, 3, 2),
]


@pytest.mark.parametrize("args", GEOMS)
def test_geometry_matches_oracle(fg, oracle, args):
    g = fg.fl_conv_geom_make(*args)
    o = oracle.geometry(*args)
    d = g.as_dict()
    for k in ("Hp", "Wp", "Ho", "Wo", "Rin", "Rout", "bands", "P", "c_n", "G", "n_in", "n_out"):
        assert d[k] == getattr(o, k), k
    assert (d["stride"], d["pad"]) == (o.s, o.p)


def test_geometry_rejects_bad_shapes(fg):
    for args in [(4096, 0, 1, 4, 4, 3, 1, 1), (4095, 1, 1, 4, 4, 3, 1, 1), (4096, 1, 1, 2, 2, 5, 1, 0),
                 (64, 1, 1, 40, 40, 3, 1, 1)]:
        with pytest.raises(fg.FlashError):
            fg.fl_conv_geom_make(*args)
