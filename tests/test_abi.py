"""The C ABI on a machine without a GPU: the library builds, loads, exports every function the
header declares, and rejects invalid problem definitions before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2501_17913_gb300 import build as B
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tjm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s+\**(tjm_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return tjm.load()


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert len(names) >= 25, names
    raw = C.CDLL(B.LIB)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    # and the binding marshals every one of them except the device-pointer SVD entry point
    bound = {n for n, _, _ in tjm.SIGNATURES}
    assert set(names) - bound <= {"tjm_svd_noalloc"}, set(names) - bound


def test_default_options(lib):
    o = tjm.tjm_options()
    lib.tjm_default_options(C.byref(o))
    assert (o.precision, o.krylov_max, o.krylov_tol, o.exact_full_bond, o.device, o.max_ctas) == \
           (tjm.PREC_FP32_DF64, 30, 0.0, 0, 0, 0)
    assert (o.energy_shift, o.tile_rule, o.tensor_cores, o.trotter_order, o.projection_error) == (1, 0, 0, 2, 0)


@pytest.mark.parametrize("case", ["dt", "chi_low", "chi_high", "eps", "one_site", "open_end", "precision",
                                  "tile_rule"])
def test_invalid_problems_rejected_before_any_device_call(lib, case):
    """These checks come first in tjm_create, so they return TJM_EINVAL even where no GPU exists."""
    W, dt, chi, eps, kw = I.xxx_mpo(4, 1.0, 0.5), 0.1, 8, 1e-10, {}
    if case == "dt":
        dt = 0.0
    elif case == "chi_low":
        chi = 0
    elif case == "chi_high":
        chi = 65
    elif case == "eps":
        eps = -1e-3
    elif case == "one_site":
        W = [np.eye(2, dtype=complex).reshape(1, 1, 2, 2)]
    elif case == "open_end":
        W = list(W[:-1]) + [np.concatenate([W[-1], W[-1]], axis=1)]     # last right bond 2, not 1
    elif case == "precision":
        kw = {"precision": 7}
    elif case == "tile_rule":
        kw = {"tile_rule": 2}
    with pytest.raises(tjm.TJMError) as e:
        tjm.Context(W, I.noise(len(W), 0.1, 0.1), dt, chi, eps, **kw)
    assert e.value.status == tjm.TJM_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's sizes and field offsets (a C program
    compiled against include/tjm.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"tjm_mpo": tjm.tjm_mpo, "tjm_jump": tjm.tjm_jump, "tjm_observable": tjm.tjm_observable,
               "tjm_observable2": tjm.tjm_observable2,
               "tjm_state": tjm.tjm_state, "tjm_options": tjm.tjm_options, "tjm_stats": tjm.tjm_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tjm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        got = C.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_complex_marshalling_is_interleaved_row_major():
    """Operators and states cross the ABI as interleaved (re, im) doubles, row-major (tjm.h)."""
    op = np.array([[1 + 2j, 3 - 4j], [5j, -6.0]])
    assert list(tjm._op8(op)) == [1, 2, 3, -4, 0, 5, -6, 0]
    site = np.arange(12).reshape(2, 2, 3) * (1 + 1j)
    flat = tjm._cplx(site)
    assert flat.shape == (24,) and np.array_equal(flat[0::2], site.real.ravel()) and \
        np.array_equal(flat[1::2], site.imag.ravel())
