"""Host-side checks that need no GPU: the library builds, loads and exports
every symbol declared in include/kx.h, and the header matches the binding."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+([a-zA-Z_][a-zA-Z_0-9]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["krylov_expm_create", "krylov_expm_destroy", "apply_A", "arnoldi", "expm_phi_project",
              "stationary_solve", "response_at_freqs"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1707_00023_gb300 import _binding
    if not os.path.exists(_binding.LIBPATH):
        from paper_1707_00023_gb300 import build
        build.build()
    lib = ctypes.CDLL(_binding.LIBPATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(_binding.EXPORTS) == declared_functions()


def test_binding_refuses_missing_library(tmp_path):
    from paper_1707_00023_gb300 import _binding
    with pytest.raises(RuntimeError):
        _binding.load_library(str(tmp_path / "nope.so"))


def test_create_without_gpu_reports_error():
    """On a host without a GPU the ABI returns an error code, never aborts."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    from paper_1707_00023_gb300 import _binding
    lib = _binding.load_library()
    d = _binding.Desc()
    d.dim = 2
    d.n = (ctypes.c_int * 3)(8, 8, 1)
    d.bc = (ctypes.c_int * 3)(1, 1, 0)
    d.layer_axis = 0
    d.layer_cells = 2
    d.sigma_max = 1.0
    d.precision = 0
    d.krylov_dim = 8
    d.max_freqs = 1
    d.batch = 1
    eps = (ctypes.c_double * 64)(*([1.0] * 64))
    h = ctypes.c_void_p()
    st = lib.krylov_expm_create(ctypes.byref(d), eps, None, ctypes.byref(h))
    assert st != 0
    assert lib.kx_last_error(None)
    # descriptor validation happens before any device call
    d.krylov_dim = 1000
    assert lib.krylov_expm_create(ctypes.byref(d), eps, None, ctypes.byref(h)) == _binding.KX_EINVAL


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the size and field
    offsets the C compiler gives the header's declaration."""
    import shutil
    import subprocess
    from paper_1707_00023_gb300 import _binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"kx_desc": B.Desc, "kx_stats": B.Stats, "kx_batch_info": B.BatchInfo,
               "kx_kernel_time": B.KernelTime}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
