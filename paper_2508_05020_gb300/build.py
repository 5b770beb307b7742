"""Build libamr (the CUDA library behind include/amr.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel and linked into
``paper_2508_05020_gb300/_lib/libamr.so``. The FP64 kernel unit is compiled
with -fmad=false so that its arithmetic is one IEEE rounding per operation.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, '_lib')
LIB = os.path.join(OUT, 'libamr.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
COMMON = ['-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC', '-Xcompiler', '-ffp-contract=off',
          '-I', CSRC, '-I', os.path.join(ROOT, 'include')]
UNITS = {
    'amr_f64.cu': ['-fmad=false'],
    'amr_f32.cu': ['-prec-sqrt=false'],
    'amr_common.cu': [],
    'amr_api.cu': [],
    'amr_mesh.cpp': [],
    'amr_mlp.cu': [],
}


def nvcc():
    for p in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc'):
        if p and os.path.exists(p):
            return p
    return 'nvcc'


def _compile(src, extra, verbose):
    obj = os.path.join(OUT, src + '.o')
    cmd = [nvcc()] + ARCH + COMMON + extra + ['-c', os.path.join(CSRC, src), '-o', obj]
    if verbose:
        cmd.insert(1, '-Xptxas=-v')
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed on %s:\n%s\n%s' % (src, r.stdout, r.stderr))
    return obj, r.stderr


def sources_newer_than(path):
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    for d in (CSRC, os.path.join(ROOT, 'include')):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return os.path.getmtime(__file__) > t


def build(force=False, verbose=False, jobs=None):
    """Compile and link libamr.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    if not force and not sources_newer_than(LIB):
        return LIB
    with cf.ThreadPoolExecutor(max_workers=jobs or len(UNITS)) as ex:
        futs = [ex.submit(_compile, s, e, verbose) for s, e in UNITS.items()]
        objs = []
        for f in futs:
            obj, log = f.result()
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = LIB + '.tmp'
    cmd = [nvcc()] + ARCH + ['-shared', '-o', tmp] + objs + ['-lcudart']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose='-v' in sys.argv))
