"""In-tree build of libmgfld.so for sm_103a (nvcc, no cmake).

Each CUDA translation unit is compiled in parallel, then linked into
paper_1809_05608_gb300/_build/libmgfld.so.  Objects are rebuilt only when a
source or header is newer than the object."""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(BUILD, 'libmgfld.so')

SOURCES = ['setup.cu', 'assemble.cu', 'blocktri.cu', 'step.cu', 'noalloc.cu', 'adjoint.cu', 'eadvect.cu',
           'stress.cu', 'pair.cu', 'check.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
NVCC_FLAGS = ARCH + ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC,-O2',
                     '-I', INCLUDE, '-I', CSRC]


def _nvcc():
    exe = shutil.which('nvcc')
    if exe is None and os.path.exists('/usr/local/cuda/bin/nvcc'):
        exe = '/usr/local/cuda/bin/nvcc'
    if exe is None:
        raise RuntimeError('nvcc not found: the CUDA toolkit is required to build libmgfld')
    return exe


def _headers():
    hs = [os.path.join(INCLUDE, 'mgfld.h')]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(('.cuh', '.h'))]
    return hs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libmgfld.so; returns its path.  Raises on any compiler error."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = _headers()
    objs = []
    cmds = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace('.cu', '.o'))
        objs.append(o)
        if _stale(o, [s] + headers):
            cmds.append([nvcc] + NVCC_FLAGS + ['-c', s, '-o', o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError('nvcc failed:\n' + ' '.join(cmd) + '\n' + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        list(ex.map(run, cmds))
    if cmds or _stale(LIB, objs):
        run([nvcc] + ARCH + ['-shared', '-o', LIB] + objs)
    return LIB


if __name__ == '__main__':
    print(build(verbose=True))
