"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point that include/*.h declares; the product never imports the oracle;
a missing library fails loudly.  No CUDA call is made."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def libpath():
    from paper_2409_05572_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    return build_lib.LIB


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(eig_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("eig_create", "eig_solve", "eig_query", "eig_destroy", "eig_strerror",
                     "eig_spmm", "eig_gram", "eig_block_update", "eig_residual", "eig_cholqr2",
                     "eig_syev", "eig_hl_trick", "eig_convert", "eig_options_default"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.eig_strerror.restype = ctypes.c_char_p
    assert lib.eig_strerror(0) == b"ok"
    assert b"invalid" in lib.eig_strerror(1)


def test_binding_exports_match_library(libpath):
    from paper_2409_05572_gb300 import _lib
    lib = _lib.load()
    for name in _lib.EXPORTS:
        assert hasattr(lib, name)
    assert set(_lib.EXPORTS) <= declared_functions()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2409_05572_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2409_05572_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        src = open(path, errors="ignore").read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), path
        assert "oracle/" not in src, path


def test_options_default_values(libpath):
    from paper_2409_05572_gb300 import _lib
    lib = _lib.load()
    o = _lib.eig_options()
    assert lib.eig_options_default(ctypes.byref(o)) == 0
    assert (o.tol, o.max_iter, o.je, o.js, o.jp, o.j_warm) == (1e-10, 1000, 12, 2, 10, 5)
    assert (o.mu, o.r_warm, o.cheb_degree) == (1.1, 1e-4, 12)
    assert (o.expand_powered, o.gram_tc, o.warm_first, o.expand_random, o.seed) == (0, 1, 0, 0, 0)
    assert o.tc_chunk_rows == 0


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's field offsets
    and sizes (compiled with the host C compiler)."""
    import shutil
    import subprocess
    from paper_2409_05572_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [_lib.eig_csr, _lib.eig_options, _lib.eig_result, _lib.eig_server_opts]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "eig_gb300.h"', "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in S._fields_:
            cname = f[0].rstrip("_")   # Python keywords carry a trailing underscore
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {cname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.splitlines())
    for S in structs:
        name = S.__name__
        assert int(out[name]) == ctypes.sizeof(S), name
        for f in S._fields_:
            assert int(out[f"{name}.{f[0]}"]) == getattr(S, f[0]).offset, (name, f[0])


def test_footprint_orders_the_configurations(libpath):
    """eig_footprint (host arithmetic only): the tensor-core slice buffers
    cost memory, the c4 graph workload only fits the 280 GB of HBM without
    them, and the footprint grows with n and k_max."""
    from paper_2409_05572_gb300 import _lib
    _lib.load()
    f = _lib.footprint
    c2 = f(2_097_152, 14_581_760, 64, 128)
    assert 60e9 < c2 < 100e9
    assert f(2_097_152, 14_581_760, 64, 128, gram_tc=0) < c2
    c4 = dict(precond=1, deflate_ones=1)
    assert f(4_000_000, 44_000_000, 200, 400, **c4) > 280e9 > f(4_000_000, 44_000_000, 200, 400, gram_tc=0, **c4)
    # row-chunked slice buffers bring the tensor-core products back under HBM
    chunked = [f(4_000_000, 44_000_000, 200, 400, tc_chunk_rows=r, **c4) for r in (262_144, 1_048_576)]
    assert f(4_000_000, 44_000_000, 200, 400, gram_tc=0, **c4) < chunked[0] < chunked[1] < 280e9
    sizes = [f(n, 7 * n, 32, k) for n in (10_000, 100_000, 1_000_000) for k in (64, 96, 128)]
    assert sizes == sorted(sizes[:3]) + sorted(sizes[3:6]) + sorted(sizes[6:])
    for k in range(3):
        assert sizes[k] < sizes[3 + k] < sizes[6 + k]


def test_norm_bound_is_the_gershgorin_bound(libpath):
    """eig_norm_bound (host only): max_i sum_j |a_ij|, an upper bound of
    ||A||_2 -- exact for the 2D Dirichlet Laplacian's interior rows (8), close
    for the Anderson Hamiltonian, within 2x for a graph Laplacian; float32
    values give the same bound; device or malformed CSR is rejected."""
    import numpy as np
    from paper_2409_05572_gb300 import _lib
    from paper_2409_05572_gb300 import workloads as W
    _lib.load()
    for A in (W.laplacian_2d(16), W.anderson_3d(6, seed=2), W.graph_laplacian(2000, seed=3)):
        M = A.to_scipy()
        want = float(np.max(np.asarray(abs(M).sum(axis=1)).ravel()))
        got = _lib.norm_bound(A)
        assert abs(got - want) <= 1e-14 * want   # the same sums, in row order
        norm2 = float(np.max(np.abs(np.linalg.eigvalsh(M.toarray()))))
        assert norm2 <= got * (1 + 1e-12) and got <= 2.0 * norm2 + 1e-12
        A32 = W.CSR(A.n, A.indptr, A.indices, A.data.astype(np.float32))
        assert abs(_lib.norm_bound(A32) - want) <= 1e-6 * want
    assert _lib.norm_bound(W.laplacian_2d(16)) == 8.0
    bad = W.laplacian_2d(4)
    bad = W.CSR(bad.n, np.concatenate([[1], bad.indptr[1:]]).astype(np.int32), bad.indices, bad.data)
    with pytest.raises(_lib.EigError):
        _lib.norm_bound(bad)
