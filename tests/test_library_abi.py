"""The C-ABI library builds, loads and exports every symbol include/ewave.h declares.
No compute calls: these run without a GPU."""
import os
import re
import subprocess
import sys

import pytest


def _declared(repo_root):
    txt = open(os.path.join(repo_root, "include", "ewave.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ewv_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib(repo_root):
    so = os.path.join(repo_root, "paper_2401_16322_gb300", "libewave.so")
    if not os.path.exists(so):
        subprocess.run([sys.executable, "-m", "paper_2401_16322_gb300.build"], cwd=repo_root,
                       check=True)
    from paper_2401_16322_gb300 import ewave
    return ewave.load_library()


def test_header_declarations_match_binding(repo_root):
    from paper_2401_16322_gb300 import ewave
    assert _declared(repo_root) == sorted(ewave.EXPORTS)


def test_library_exports_every_declared_symbol(lib, repo_root):
    for name in _declared(repo_root):
        assert hasattr(lib, name), name


def test_version_string(lib):
    assert b"sm_103a" in lib.ewv_version()


def test_null_handle_errors_without_gpu(lib):
    # argument checks happen before any CUDA call
    import ctypes
    assert lib.ewv_destroy_model(None) == -1
    assert lib.ewv_set_stream(None, None) == -1
    assert lib.ewv_last_error(None) == b"null handle"
    assert lib.ewv_create_model(None, None) == -1
    assert lib.ewv_step_krylov_dense(None, 0.0, 1e-3, 8, None) == -1
    assert lib.ewv_adjoint_step_krylov_dense(None, 0.0, 1e-3, 8, None, None, None) == -1
    assert lib.ewv_adjoint_step(None, 0, 0.0, 1e-3, 8, None, None, None) == -1


def test_checkpoint_stride_host_logic_matches_oracle(lib):
    # pure host arithmetic in the library: bit-exact against the oracle's schedule
    import ctypes
    from oracle.adjoint import checkpoint_stride as o_stride
    out = ctypes.c_int()
    for n in range(0, 60):
        for b in range(1, 25):
            assert lib.ewv_checkpoint_stride(n, b, ctypes.byref(out)) == 0
            assert out.value == o_stride(n, b), (n, b)
    assert lib.ewv_checkpoint_stride(-1, 4, ctypes.byref(out)) == -1
    assert lib.ewv_checkpoint_stride(10, 0, ctypes.byref(out)) == -1
    assert lib.ewv_checkpoint_stride(10, 4, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    # the binding has no fallback: without the built library every entry point raises
    from paper_2401_16322_gb300 import ewave
    saved = ewave._lib
    ewave._lib = None
    try:
        with pytest.raises(ewave.EwaveError, match="missing"):
            ewave.load_library(str(tmp_path / "libewave.so"))
    finally:
        ewave._lib = saved


def test_create_model_rejects_bad_extents_without_gpu(lib):
    # descriptor checks return before any CUDA call
    import ctypes
    from paper_2401_16322_gb300 import ewave
    base = dict(dims=2, nx=64, ny=32, dx=10.0, fd_order=8, pml_width=4, beta0=10.0,
                free_surface=1, precision=0, nshots=1, src_taylor_p=8, max_receivers=4, nz=1)
    out = ctypes.c_void_p()
    for bad in (dict(nx=1), dict(ny=(1 << 30) + 1), dict(nx=2 ** 31 - 1),
                dict(dims=3, nz=(1 << 30) + 1), dict(dims=3, nz=1), dict(dims=4),
                dict(src_taylor_p=0), dict(fd_order=6), dict(dx=0.0), dict(nshots=0)):
        d = ewave.ModelDesc(**{**base, **bad})
        assert lib.ewv_create_model(ctypes.byref(d), ctypes.byref(out)) == -1, bad
        assert not out.value


def test_oracle_and_product_share_no_code(repo_root):
    # the product package never imports the oracle, and the oracle imports nothing of the
    # product (the seeded input generator is imported by the tests, not by oracle/)
    import ast
    import glob

    def imported(path):
        tree = ast.parse(open(path).read())
        names = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names.update(a.name.split(".")[0] for a in node.names)
            elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
                names.add(node.module.split(".")[0])
        return names

    for p in glob.glob(os.path.join(repo_root, "paper_2401_16322_gb300", "*.py")):
        assert "oracle" not in imported(p), p
    for p in glob.glob(os.path.join(repo_root, "oracle", "*.py")):
        assert "paper_2401_16322_gb300" not in imported(p), p


def test_oracle_is_used_only_by_smoke_and_the_cpu_baseline(repo_root):
    # outside tests/, only __graft_entry__.smoke() and bench.py's CPU-baseline sampler (used
    # by the cpu_baseline figure and the reference arm) import the oracle
    import ast

    def users(path):
        tree = ast.parse(open(path).read())
        out = set()
        for fn in ast.walk(tree):
            if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
                for node in ast.walk(fn):
                    mod = (node.module if isinstance(node, ast.ImportFrom) else
                           node.names[0].name if isinstance(node, ast.Import) else None)
                    if mod and mod.split(".")[0] == "oracle":
                        out.add(fn.name)
        top = {n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))}
        assert not any((getattr(n, "module", None) or n.names[0].name).split(".")[0] == "oracle"
                       for n in top), path
        return out

    assert users(os.path.join(repo_root, "__graft_entry__.py")) == {"smoke"}
    assert users(os.path.join(repo_root, "bench.py")) == {"_oracle_worker", "sample", "_oracle_full_worker",
                                                          "oracle_full_runs"}
