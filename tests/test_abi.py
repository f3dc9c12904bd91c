"""C-ABI checks that need no GPU: the library loads, exports every function
``include/fs.h`` declares, and rejects bad arguments on the host (FS_EINVAL,
with a message) before launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1810_10496_gb300 import build
    build.build()
    import paper_1810_10496_gb300 as fs
    return fs.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "fs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fs_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"fs_normalize", "fs_build_db", "fs_knn", "fs_recommend", "fs_workspace_size",
            "fs_db_destroy", "fs_last_error"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_no_oracle_in_product():
    """The product path must not import or call the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_1810_10496_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn


def test_host_validation(L):
    import paper_1810_10496_gb300 as fs
    P = ctypes.c_void_p
    fake = P(0x1000)     # never dereferenced: every call below fails its host checks
    # NULL database
    assert L.fs_knn(None, fake, 1, None, None, None, fake, 1 << 20, fake, fake, None) == fs.FS_EINVAL
    assert "db" in fs.fs_last_error()
    assert L.fs_recommend(None, fake, 1, None, None, None, fake, 1, fake, fake, fake, fake, 8,
                          None, None) == fs.FS_EINVAL
    # normalize: f out of range, ld < f, negative n, NULL pointers
    assert L.fs_normalize(fake, 4, 0, 4, fake, None, None) == fs.FS_EINVAL
    assert L.fs_normalize(fake, 4, 2000, 2000, fake, None, None) == fs.FS_EINVAL
    assert L.fs_normalize(fake, 4, 8, 4, fake, None, None) == fs.FS_EINVAL
    assert "ld" in fs.fs_last_error()
    assert L.fs_normalize(fake, -1, 8, 8, fake, None, None) == fs.FS_EINVAL
    assert L.fs_normalize(None, 3, 8, 8, fake, None, None) == fs.FS_EINVAL
    assert L.fs_normalize(None, 0, 8, 8, None, None, None) == fs.FS_OK   # nothing to do
    # build: bad precision, out NULL, f too large for the tensor-core scans,
    # malformed segment offsets (host array)
    out = P()
    assert L.fs_build_db(fake, 10, 8, fake, fake, None, 1, 7, None, ctypes.byref(out)) == fs.FS_EINVAL
    assert L.fs_build_db(fake, 10, 8, fake, fake, None, 1, 0, None, None) == fs.FS_EINVAL
    assert L.fs_build_db(fake, 10, 300, fake, fake, None, 1, 1, None, ctypes.byref(out)) == fs.FS_EINVAL
    assert "f=300" in fs.fs_last_error()
    segs = np.array([0, 5, 3, 10], dtype=np.int64)
    assert L.fs_build_db(fake, 10, 8, fake, fake, segs.ctypes.data, 3, 0, None,
                         ctypes.byref(out)) == fs.FS_EINVAL
    segs = np.array([0, 5, 9], dtype=np.int64)
    assert L.fs_build_db(fake, 10, 8, fake, fake, segs.ctypes.data, 2, 0, None,
                         ctypes.byref(out)) == fs.FS_EINVAL
    assert L.fs_build_db(fake, -2, 8, fake, fake, None, 1, 0, None, ctypes.byref(out)) == fs.FS_EINVAL
    assert not out.value
    # other entry points with NULL handles
    sz = ctypes.c_size_t()
    assert L.fs_workspace_size(None, 4, None, ctypes.byref(sz)) == fs.FS_EINVAL
    assert L.fs_db_destroy(None) == fs.FS_EINVAL
    assert L.fs_db_check(None, None) == fs.FS_EINVAL
    assert L.fs_db_stats(None, None, 0, None) == fs.FS_EINVAL


def test_binding_names_match_header():
    import paper_1810_10496_gb300 as fs
    for n in _declared():
        assert hasattr(fs, n), n
