"""The C-ABI library builds, loads and exports every symbol that
include/sfmm.h declares (CPU only: no CUDA compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_05804_gb300 import build

    return ctypes.CDLL(build.build())


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sfmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sfmm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_2602_05804_gb300 import sfmm

    assert sorted(sfmm.EXPORTS) == declared_functions()


def test_strerror_and_version_without_gpu(lib):
    from paper_2602_05804_gb300 import sfmm

    sfmm.load()
    assert sfmm.sfmm_strerror(sfmm.SFMM_ECAPACITY) == "work buffer capacity exceeded"
    assert sfmm.sfmm_strerror(12345) == "unknown error"
    assert sfmm.sfmm_version().startswith("sfmm-gb300")


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2602_05804_gb300 import sfmm

    with pytest.raises(ImportError):
        sfmm._lib_saved = sfmm._lib
        sfmm._lib = None
        try:
            sfmm.load(str(tmp_path / "missing.so"))
        finally:
            sfmm._lib = sfmm._lib_saved


def test_generated_expansion_is_current():
    """The committed generated header equals the generator's output."""
    import subprocess
    import sys

    path = os.path.join(ROOT, "paper_2602_05804_gb300", "csrc", "expansion_gen.cuh")
    before = open(path).read()
    subprocess.run([sys.executable, os.path.join(os.path.dirname(path), "gen_expansion.py")], check=True,
                   stdout=subprocess.DEVNULL)
    assert open(path).read() == before
