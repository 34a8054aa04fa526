"""CPU checks of the boundary: the library builds, loads without a GPU, and exports every
function include/rgbd_lbp.h declares; the binding wraps each of them under the same name."""
import ctypes
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_01883_gb300 import _build
    return _build.build()


def test_header_declares_the_four_calls():
    from paper_1504_01883_gb300 import binding
    names = binding.declared_functions()
    for call in ["rgbd_crop_affine", "lbp_fused_features", "svm_train_data_pack", "svm_score"]:
        assert call in names
    assert len(names) >= 12


def test_library_exports_every_declared_symbol(built_lib):
    from paper_1504_01883_gb300 import binding
    L = ctypes.CDLL(built_lib)
    for name in binding.declared_functions():
        assert hasattr(L, name), name
    assert L.rgbd_version() == (1 << 16)


def test_binding_names_match_header():
    import paper_1504_01883_gb300.binding as b
    for call in ["rgbd_crop_affine", "lbp_fused_features", "lbp_normalize_features", "svm_train_data_pack",
                 "svm_score"]:
        assert callable(getattr(b, call))


def test_errors_are_reported_without_a_gpu(built_lib):
    """Argument checks run before any CUDA call: a NULL context is rejected with a message."""
    from paper_1504_01883_gb300 import binding
    L = binding.lib()
    rc = L.lbp_fused_features(None, None, None, 0, 0, 0, None, None, 1, 128, 8, 150, 0, None, 0, None, 0,
                              ctypes.c_float(1.0), None, None, None)
    assert rc == -1
    assert "ctx" in binding.last_error()
    rc = L.svm_score(None, None, None, None, 0, ctypes.c_float(1.0), None, None, None)
    assert rc == -1
    out = ctypes.c_void_p()
    assert L.rgbd_server_create(None, None, ctypes.byref(out)) == -1
    assert "rgbd_server_create" in binding.last_error()


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_1504_01883_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.lib()


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1504_01883_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "rgbd_oracle" not in text, f
