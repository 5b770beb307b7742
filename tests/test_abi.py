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


C_PROGRAM = r'''
#include "amr.h"
#include <stdio.h>
int main(void) {
    amr_options_t o;
    int base[3] = {4, 4, 1}, per[3] = {0, 0, 0}, keys[16 * 4], out[64 * 4], n_out = 0, i, rc;
    int req[4] = {0, 1, 1, 0};
    amr_default_options(&o);
    for (i = 0; i < 16; ++i) {
        keys[4 * i] = 0; keys[4 * i + 1] = i % 4; keys[4 * i + 2] = i / 4; keys[4 * i + 3] = 0;
    }
    rc = amr_mesh_close(2, base, per, 2, 16, keys, 1, req, 0, NULL, 64, &n_out, out, NULL, NULL);
    printf("%d %d %d %.2f\n", rc, n_out, o.precision, o.cfl);
    return rc;
}
'''


def test_header_is_plain_c_and_links(libpath, tmp_path):
    # include/amr.h compiles as strict C99 and a C program links against the
    # library and calls it (host-only entry points: no GPU needed)
    import shutil
    if not shutil.which('gcc'):
        pytest.skip('no C compiler')
    src = tmp_path / 't.c'
    src.write_text(C_PROGRAM)
    exe = tmp_path / 't'
    libdir = os.path.dirname(libpath)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(shutil.which('nvcc') or
                                                                              '/usr/local/cuda/bin/nvcc'))), 'lib64')
    r = subprocess.run(['gcc', '-std=c99', '-Wall', '-Wextra', '-pedantic', '-Werror', '-I', os.path.join(ROOT, 'include'),
                        str(src), '-L', libdir, '-lamr', '-Wl,-rpath,' + libdir, '-Wl,-rpath-link,' + cuda_lib,
                        '-o', str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=cuda_lib + os.pathsep + os.environ.get('LD_LIBRARY_PATH', ''))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env)
    assert r.returncode == 0 and r.stdout.split() == ['0', '20', '64', '0.50'], (r.stdout, r.stderr)
