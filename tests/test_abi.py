"""The C-ABI library builds and exports every function include/nolsm.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nolsm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(nolsm_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2205_12182_gb300.build import build
    return build()


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["nolsm_build_submatrices", "nolsm_sign_batch", "nolsm_set_mu", "nolsm_density", "nolsm_band_energy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    from paper_2205_12182_gb300 import nolsm
    assert set(nolsm.FUNCTIONS) == set(declared_functions())
    for n in nolsm.FUNCTIONS:
        assert callable(getattr(nolsm, n))


def test_options_defaults_without_gpu(lib_path):
    from paper_2205_12182_gb300 import nolsm
    o = nolsm.nolsm_default_options()
    assert o.precision == nolsm.PREC_MIXED_FP16 and o.max_iter == 100 and o.spin_factor == 2.0


def test_struct_layout_matches_c(lib_path, tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's offsetof."""
    import shutil
    import subprocess
    from paper_2205_12182_gb300 import nolsm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"nolsm_csr": nolsm.NolsmCsr, "nolsm_options": nolsm.NolsmOptions,
               "nolsm_sign_stats": nolsm.NolsmSignStats, "nolsm_chunked_stats": nolsm.NolsmChunkedStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nolsm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(l.split()[0], l.split()[1]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py)
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
