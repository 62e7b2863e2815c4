"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point declared in include/re.h, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re as regex

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    from paper_0812_1633_gb300 import build
    return C.CDLL(build.build())


def declared():
    src = open(os.path.join(ROOT, "include", "re.h")).read()
    src = regex.sub(r"/\*.*?\*/", "", src, flags=regex.S)
    return sorted(set(regex.findall(r"\b(re_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(so):
    names = declared()
    assert "re_create" in names and "re_lj_forces_device" in names and len(names) >= 20
    for n in names:
        assert hasattr(so, n), n


def test_library_is_built_for_sm103a():
    """The build compiles every translation unit for sm_103a only (one
    -gencode pair, no PTX for other architectures)."""
    from paper_0812_1633_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_argument_validation_without_gpu():
    import numpy as np
    import paper_0812_1633_gb300 as re
    from paper_0812_1633_gb300 import inputs
    L = inputs.box_length(256)
    bad = [
        dict(N=250, L=L, rc=2.5, temps=[1.0, 1.1]),           # not 4 k^3
        dict(N=256, L=L, rc=3.2, temps=[1.0, 1.1]),           # list radius beyond L/2
        dict(N=256, L=L, rc=2.5, temps=[1.0, 1.0]),           # duplicate temperatures
        dict(N=256, L=L, rc=2.5, temps=[1.0, -1.0]),          # negative temperature
        dict(N=256, L=L, rc=2.5, temps=[]),                   # no replicas
        dict(N=4 * 26 ** 3, L=40.0, rc=2.5, temps=[1.0]),     # N > 65535
    ]
    for kw in bad:
        with pytest.raises(re.REError) as e:
            re.Context(kw["N"], kw["L"], kw["rc"], np.array(kw["temps"], float), 1)
        assert e.value.code == re.RE_EINVAL, kw


def test_default_opts_match_paper():
    import paper_0812_1633_gb300 as re
    o = re.default_opts()
    assert o["dt"] == 0.005 and o["skin"] == 0.5   # time step 0.005, list radius 3.0 = 2.5 + 0.5
    assert o["shift_energy"] == 1 and o["precision"] == re.PREC["mixed"]


def test_header_compiles_as_c99(tmp_path):
    """include/re.h is a plain C header: it compiles with a C99 compiler on its own."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_re.c"
    src.write_text('#include "re.h"\n'
                   "int main(void) { size_t n = 0; re_opts o; re_default_opts(&o);\n"
                   "  return re_checkpoint_size(0, &n) == RE_OK; }\n")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-c", str(src), "-o", str(tmp_path / "use_re.o")])
