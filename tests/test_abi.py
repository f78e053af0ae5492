"""The C ABI: every declared entry point is exported, and host-side argument
checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1005_5405_gb300 import binding, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "bz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bz_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1005_5405_gb300 import build
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.exported_symbols()) == set(names)


def test_version(lib):
    assert b"sm_103a" in lib.bz_version()


def test_argument_validation_without_gpu(lib):
    def create(**kw):
        p = workloads.small(**kw)
        try:
            binding.Cavity(p)
        except binding.BzError as e:
            return e.status, str(e)
        return 0, ""
    assert create(nt=0)[0] == binding.BZ_EINVAL
    assert create(nv=1)[0] == binding.BZ_EINVAL
    assert create(nx=0)[0] == binding.BZ_EINVAL
    assert create(kn=-1.0)[0] == binding.BZ_EINVAL
    assert create(cfl=1.5)[0] == binding.BZ_EINVAL
    assert create(lid_period=-1.0)[0] == binding.BZ_EINVAL
    # Batches run the shared sample set only (checked before any device work).
    with pytest.raises(binding.BzError) as e:
        binding.Batch([workloads.small(per_cell=True)])
    assert e.value.status == binding.BZ_EUNSUPPORTED and "shared sample set" in str(e.value)


def test_allocation_fault_injection(lib):
    os.environ["BZ_FAULT"] = "alloc"
    try:
        with pytest.raises(binding.BzError) as e:
            binding.Cavity(workloads.small())
        assert e.value.status == binding.BZ_ENOMEM
    finally:
        del os.environ["BZ_FAULT"]


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.bz_create(None, None, None, None, C.byref(h)) == binding.BZ_EINVAL
    assert lib.bz_step(None, 1, None) == binding.BZ_EINVAL
    assert lib.bz_destroy(None) == binding.BZ_OK
    assert b"NULL" in lib.bz_last_error() or lib.bz_last_error() != b""
