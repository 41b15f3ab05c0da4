"""The in-tree build recompiles a translation unit only when one of its own
dependencies (from the .d file nvcc writes) is newer than its object."""
import os

from paper_2101_04550_gb300 import build


def _touch(path, t):
    with open(path, "a"):
        pass
    os.utime(path, (t, t))


def test_dependency_file_parsing(tmp_path):
    dep = tmp_path / "x.d"
    dep.write_text("_build/x.o : csrc/x.cu \\\n    csrc/a.cuh \\\n    /usr/include/stdio.h\n")
    assert build._deps(str(dep)) == ["csrc/x.cu", "csrc/a.cuh", "/usr/include/stdio.h"]
    assert build._deps(str(tmp_path / "missing.d")) is None


def test_stale_follows_own_dependencies(tmp_path):
    # every time here lies after the build script's own (also a dependency)
    t0 = os.path.getmtime(build.__file__) + 1000
    src, hdr, other = tmp_path / "x.cu", tmp_path / "a.cuh", tmp_path / "b.cuh"
    obj, dep = tmp_path / "x.o", tmp_path / "x.d"
    for p in (src, hdr, other):
        _touch(p, t0)
    dep.write_text(f"{obj} : {src} {hdr}\n")
    _touch(obj, t0 + 50)
    assert not build._stale(str(src), str(obj))
    _touch(other, t0 + 100)     # not a dependency of x.o
    assert not build._stale(str(src), str(obj))
    _touch(hdr, t0 + 100)       # a dependency
    assert build._stale(str(src), str(obj))
    _touch(obj, t0 + 150)
    os.remove(dep)              # no dependency file: rebuild
    assert build._stale(str(src), str(obj))
