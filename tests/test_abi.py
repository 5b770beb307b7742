"""The C ABI: every function declared in include/amr.h is exported by the
built library and bound by the Python layer (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, 'include', 'amr.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(amr_[a-z0-9_]+)\s*\(', src)))


@pytest.fixture(scope='module')
def libpath():
    from paper_2508_05020_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared()
    for n in ('amr_init', 'amr_step', 'amr_regrid', 'amr_get_level', 'amr_get_diag', 'amr_set_state',
              'amr_destroy', 'amr_last_error'):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(['nm', '-D', '--defined-only', libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r'\sT\s(amr_[a-z0-9_]+)', out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2508_05020_gb300 import amr
    lib = amr.load()
    bound = {name for name, _, _ in amr.SIGNATURES}
    assert set(declared()) <= bound
    for n in declared():
        assert getattr(lib, n) is not None


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2508_05020_gb300 import amr
    monkeypatch.setattr(amr, '_lib', None)
    monkeypatch.setattr(amr, 'LIB_PATH', str(tmp_path / 'nope.so'))
    with pytest.raises(ImportError):
        amr.load()
