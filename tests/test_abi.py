"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h, and its host-side checks (configuration rules, null handles,
batch and server arguments, checkpoint states) reject bad input before any
device work (no device calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(mr_[a-z_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1905_08717_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mr_create", "mr_adapt", "mr_step", "mr_read", "mr_destroy", "mr_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_config_is_rejected_without_device_work(lib):
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.burgers_1d(L=6)
    bad = p.replace(rk_order=4)
    cfg = pkg.make_config(bad)
    h = ctypes.c_void_p()
    lib.mr_create.argtypes = [ctypes.POINTER(pkg.mr_config), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    r = lib.mr_create(ctypes.byref(cfg), q.ctypes.data, None, ctypes.byref(h))
    assert r == 1 and not h.value
    lib.mr_last_error.restype = ctypes.c_char_p
    assert lib.mr_last_error(None) == b"null handle"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1905_08717_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.library()


_BAD = {
    "dim 0": dict(dim=0), "dim 4": dict(dim=4),
    "max_level 0": dict(max_level=0), "max_level above 16": dict(max_level=17),
    "3D L=11 (2^33 cells)": dict(dim=3, max_level=11, min_level=2),
    "min_level -1": dict(min_level=-1), "min_level above max": dict(min_level=7),
    "equation -1": dict(equation=-1), "equation 4": dict(equation=4),
    "rk 1": dict(rk_order=1), "rk 4": dict(rk_order=4),
    "time mode 2": dict(time_mode=2), "precision 2": dict(precision=2),
    "AUSM+ for Burgers": dict(flux=1), "flux 2": dict(flux=2),
    "adapt mode 3": dict(adapt_mode=3),
    "cfl 0": dict(cfl=0.0), "cfl NaN": dict(cfl=float("nan")),
    "eps < 0": dict(eps=-1e-3), "eps NaN": dict(eps=float("nan")),
    "empty box": dict(hi=(0.0, 1.0, 1.0)), "wall type 3": dict(bc=(3, 0, 0)),
}


@pytest.mark.parametrize("name", sorted(_BAD))
def test_every_invalid_config_is_rejected_before_device_work(lib, name):
    """validate() runs before any CUDA call: each rule rejects on a host
    without a GPU, and no handle is returned."""
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.burgers_1d(L=6)
    cfg = pkg.make_config(p.replace(**_BAD[name]))
    h = ctypes.c_void_p()
    lib.mr_create.argtypes = [ctypes.POINTER(pkg.mr_config), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    assert lib.mr_create(ctypes.byref(cfg), q.ctypes.data, None, ctypes.byref(h)) == 1
    assert not h.value


def test_euler_specific_rules(lib):
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.euler_1d_sod(L=6)
    lib.mr_create.argtypes = [ctypes.POINTER(pkg.mr_config), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    for bad in (dict(bc=(inputs.BC_DIRICHLET0,) * 3), dict(phys=(1.0,) + (0.0,) * 7)):
        h = ctypes.c_void_p()
        cfg = pkg.make_config(p.replace(**bad))
        assert lib.mr_create(ctypes.byref(cfg), q.ctypes.data, None, ctypes.byref(h)) == 1, bad
        assert not h.value


def test_null_handles_and_arguments(lib):
    """Every entry point checks its handle and arguments on the host."""
    vp = ctypes.c_void_p
    for name, args in [("mr_reset", (None, None)), ("mr_set_tree", (None, None)), ("mr_adapt", (None,)),
                       ("mr_set_async", (None, 1)), ("mr_sync", (None,)), ("mr_profile", (None, 1)),
                       ("mr_set_grid_cap", (None, 0)), ("mr_batch_set_grid_cap", (None, 0)),
                       ("mr_set_launch_mode", (None, 0)), ("mr_reserve_nodes", (None, ctypes.c_longlong(8))), ("mr_selftest_grid_wait", (0, 0, ctypes.c_double(1.0), None)),
                       ("mr_server_set_grid_cap", (None, 0)), ("mr_server_advance", (None, None, None)),
                       ("mr_server_status", (None, ctypes.c_longlong(1))),
                       ("mr_server_release", (None, ctypes.c_longlong(1)))]:
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(*args) == 1, name
    lib.mr_step.argtypes = [vp, ctypes.c_double, vp]
    lib.mr_iterate.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, vp]
    lib.mr_read.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, vp]
    lib.mr_batch_step.argtypes = [vp, ctypes.c_double, vp]
    assert lib.mr_step(None, 1.0, None) == 1
    assert lib.mr_iterate(None, 1e-3, 1, None) == 1
    assert lib.mr_read(None, 0, None, 0, None) == 1
    assert lib.mr_batch_step(None, 1.0, None) == 1
    lib.mr_launch_count.restype = ctypes.c_longlong
    assert lib.mr_launch_count(None) == 0
    lib.mr_batch_instance.restype = vp
    lib.mr_batch_instance.argtypes = [vp, ctypes.c_int]
    assert lib.mr_batch_instance(None, 0) is None
    lib.mr_server_result.restype = vp
    lib.mr_server_result.argtypes = [vp, ctypes.c_longlong]
    assert lib.mr_server_result(None, 1) is None
    lib.mr_server_memory.restype = ctypes.c_size_t
    assert lib.mr_server_memory(None) == 0
    for name in ("mr_batch_last_error", "mr_server_last_error"):
        f = getattr(lib, name)
        f.restype = ctypes.c_char_p
        assert f(None) == b"null handle"
    lib.mr_destroy(None)
    lib.mr_batch_destroy(None)
    lib.mr_server_destroy(None)


def test_batch_and_server_arguments(lib):
    import paper_1905_08717_gb300 as pkg
    vp = ctypes.c_void_p
    out, bad = vp(), ctypes.c_int(7)
    lib.mr_batch_create.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
    assert lib.mr_batch_create(0, None, None, None, ctypes.byref(out), ctypes.byref(bad)) == 1
    assert not out.value and bad.value == -1
    lib.mr_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, vp, ctypes.POINTER(vp)]
    assert lib.mr_server_create(1 << 30, 0, None, ctypes.byref(out)) == 1
    assert lib.mr_server_create(0, 4, None, ctypes.byref(out)) == 1
    assert not out.value


def test_checkpoint_state_is_checked_on_the_host(lib):
    """mr_create_from_state rejects, before any device work, a count that is
    not a macro-step boundary and keys that are not a partition of the box."""
    import numpy as np
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs
    p, _ = inputs.burgers_1d(L=3, min_level=1)
    cfg = pkg.make_config(p)
    vp = ctypes.c_void_p
    lib.mr_create_from_state.argtypes = [ctypes.POINTER(pkg.mr_config), ctypes.c_longlong, vp, vp,
                                         ctypes.c_double, ctypes.c_longlong, vp, ctypes.POINTER(vp)]

    def call(keys, iters=0):
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        vals = np.zeros(len(keys))
        out = vp()
        r = lib.mr_create_from_state(ctypes.byref(cfg), len(keys), keys.ctypes.data, vals.ctypes.data,
                                     0.0, iters, None, ctypes.byref(out))
        assert not out.value
        return r

    two = [[1, 0, 0, 0], [1, 1, 0, 0]]            # the two level-1 cells: a partition
    assert call(two, iters=3) == 5                  # 3 is not a multiple of 2^(3-1)
    assert call([[1, 0, 0, 0]]) == 1                # a hole
    assert call(two + [[2, 0, 0, 0]]) == 1          # overlapping leaves
    assert call([[0, 0, 0, 0]]) == 1                # a level below min_level
    assert call([[1, 0, 0, 0], [1, 2, 0, 0]]) == 1  # an index outside its level


@pytest.mark.parametrize("which", ["library", "oracle"])
def test_ctypes_config_matches_the_c_struct(tmp_path, which):
    """The binding's ctypes mirror of the configuration struct has the C
    compiler's field names, offsets and size (a mismatch would hand the
    library a silently corrupted configuration)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    if which == "library":
        import paper_1905_08717_gb300 as pkg
        cls, header, struct = pkg.mr_config, os.path.join(ROOT, "include", "mrlt.h"), "mr_config"
    else:
        import oracle
        cls, header, struct = oracle._Cfg, os.path.join(ROOT, "oracle", "mr_oracle.h"), "or_config"
    names = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"%s\"\nint main(void){\n"
                   "printf(\"%%zu\\n\", sizeof(%s));\n%s return 0;}\n" % (
                       header, struct,
                       "".join('printf("%%zu\\n", offsetof(%s, %s));\n' % (struct, n) for n in names)))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, n).offset for n in names]
    # every field the header declares is mirrored (a trailing field could hide in padding)
    txt = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\}" % struct, txt, flags=re.S).group(1)
    declared = [re.sub(r"\[.*?\]", "", n).strip()
                for decl in re.findall(r"\b(?:int|double)\s+([^;]+);", body) for n in decl.split(",")]
    assert declared == names


def test_readme_c_example_compiles_against_the_header(tmp_path):
    """The C usage example in the README compiles against include/mrlt.h
    (compiled only: running it needs a GPU)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    txt = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", txt, flags=re.S)
    assert blocks, "no C example in the README"
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    subprocess.run(["gcc", "-std=c99", "-D_DEFAULT_SOURCE", "-Wall", "-Werror", "-c", "-I",
                    os.path.join(ROOT, "include"), "-o", str(tmp_path / "example.o"), str(src)], check=True)
