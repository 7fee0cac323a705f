"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads
without a GPU, and exports every function include/lindblad.h declares; the
oracle and the CUDA package never import each other."""
import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lindblad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_01491_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = _declared()
    for n in ("lb_basis_create", "lb_structure_export", "lb_expand", "lb_assemble_dense",
              "lb_rk4_dense", "lb_assemble", "lb_integrate", "lb_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1912_01491_gb300 import native
    native.load()
    for n in _declared():
        assert hasattr(native._lib, n)


def test_errors_without_gpu_calls(lib):
    """Argument checks run before any CUDA call and return LB_EINVAL."""
    from paper_1912_01491_gb300 import native
    L = native.load()
    h = ctypes.c_void_p()
    assert L.lb_basis_create(1, None, ctypes.byref(h)) == native.LB_EINVAL
    assert b"N = 1" in L.lb_last_error()
    assert L.lb_basis_create(5000, None, ctypes.byref(h)) == native.LB_EINVAL
    assert L.lb_version() >= 100


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def test_oracle_and_library_are_independent():
    for d, forbidden in (("oracle", "paper_1912_01491_gb300"), ("paper_1912_01491_gb300", "oracle")):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith(".py"):
                    assert forbidden not in _imports(os.path.join(dirpath, f)), (f, forbidden)
    # the CUDA sources include nothing from the oracle and vice versa
    csrc = os.path.join(ROOT, "paper_1912_01491_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in "".join(re.findall(r'#include\s+[<"](.*?)[>"]', open(os.path.join(csrc, f)).read()))
    assert "#include \"" not in open(os.path.join(ROOT, "oracle", "lb_oracle.c")).read()


class _FakeCuda:
    """Shape, dtype and device of a CUDA tensor, without a GPU."""

    def __init__(self, shape, dtype, contiguous=True):
        import types
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = types.SimpleNamespace(type="cuda")
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for x in self.shape:
            n *= x
        return n


def test_export_buffers_checked_before_any_call():
    """structure_into's capacity is the smaller of the two buffers, and bad
    buffers raise in Python before the C entry point (and any kernel) runs."""
    torch = pytest.importorskip("torch")
    from paper_1912_01491_gb300.native import export_capacity
    i32, f64 = torch.int32, torch.float64
    assert export_capacity(_FakeCuda((10, 3), i32), _FakeCuda((12,), f64)) == 10
    assert export_capacity(_FakeCuda((12, 3), i32), _FakeCuda((7,), f64)) == 7
    bad = [
        (torch.zeros((4, 3), dtype=i32), torch.zeros(4, dtype=f64)),          # host tensors
        (_FakeCuda((4, 3), torch.int64), _FakeCuda((4,), f64)),                # wrong idx type
        (_FakeCuda((4, 3), i32), _FakeCuda((4,), torch.float32)),              # wrong val type
        (_FakeCuda((12,), i32), _FakeCuda((4,), f64)),                         # flat idx
        (_FakeCuda((4, 3), i32, contiguous=False), _FakeCuda((4,), f64)),      # strided
        (_FakeCuda((4, 3), i32), _FakeCuda((2, 2), f64)),                      # 2-D val
    ]
    for idx, val in bad:
        with pytest.raises(ValueError):
            export_capacity(idx, val)
