"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/dtsph.h declares (no GPU needed; no
compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_1904_00861_gb300 as lib_pkg
from paper_1904_00861_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dtsph.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dtsph_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def so():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ("dtsph_create", "dtsph_set_particles", "dtsph_set_boundary", "dtsph_step", "dtsph_read_field",
                 "dtsph_build_neighbors", "dtsph_get_neighbors", "dtsph_eval_rates", "dtsph_read_stats"):
        assert must in syms


def test_library_exports_every_declared_symbol(so):
    for s in declared_symbols():
        assert hasattr(so, s), s


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(lib_pkg.exported_symbols())


def test_version_and_argument_errors_without_gpu(so):
    assert lib_pkg.dtsph_version() == "0.1.0"
    # invalid parameters are rejected on the host before any CUDA call
    p = lib_pkg.make_params(dict(dim=4, h=0.1, m=0.01, nu=0.01, dt=0.01))
    with pytest.raises(lib_pkg.DtsphError) as e:
        lib_pkg.dtsph_create(p)
    assert e.value.code == -1
    p = lib_pkg.make_params(dict(dim=2, h=0.1, m=0.01, nu=0.01, dt=0.01, periodic=(1, 1, 0), hi=(0.5, 1, 1)))
    with pytest.raises(lib_pkg.DtsphError):
        lib_pkg.dtsph_create(p)       # periodic axis shorter than 9h
    p = lib_pkg.make_params(dict(dim=2, h=0.1, m=0.01, nu=0.01, dt=0.01, edac_h2_literal=1))
    with pytest.raises(lib_pkg.DtsphError) as e:
        lib_pkg.dtsph_create(p)
    assert e.value.code == -7
    for bad in (1, 9, -1):        # staging depth outside [2, 8]
        p = lib_pkg.make_params(dict(dim=2, h=0.1, m=0.01, nu=0.01, dt=0.01, lanes=1, stages=bad))
        with pytest.raises(lib_pkg.DtsphError) as e:
            lib_pkg.dtsph_create(p)
        assert e.value.code == -1
    base = dict(dim=2, h=0.1, m=0.01, nu=0.01, dt=0.01)
    for over in (dict(moving=3), dict(moving=-1), dict(moving=1, steady=1), dict(moving=1, skin=-0.1)):
        p = lib_pkg.make_params(dict(base, **over))
        with pytest.raises(lib_pkg.DtsphError) as e:
            lib_pkg.dtsph_create(p)
        assert e.value.code == -1, over
    p = lib_pkg.make_params(dict(base, moving=2))
    assert p.skin == 0.05                 # default skin h / 2
    p.skin = 0.0                          # moving = 2 needs a positive skin
    with pytest.raises(lib_pkg.DtsphError) as e:
        lib_pkg.dtsph_create(p)
    assert e.value.code == -1
    # the pair-term form, the cell size and the reused lists: bad values are
    # argument errors, unsupported combinations DTSPH_E_UNSUPPORTED (-7)
    for over, code in ((dict(form=3), -1), (dict(form=-1), -1), (dict(form=2, moving=1), -7),
                       (dict(cell_scale=0.5), -1), (dict(cell_scale=5.0), -1), (dict(list_skin=-0.01), -1),
                       (dict(list_skin=float("nan")), -1), (dict(list_skin=0.01, graph=1), -7),
                       (dict(list_skin=0.01, graph=2, shifting=1), -7), (dict(list_skin=0.01, graph=2, moving=1), -7),
                       (dict(list_skin=0.01, graph=2, steady=1), -7)):
        p = lib_pkg.make_params(dict(base, **over))
        with pytest.raises(lib_pkg.DtsphError) as e:
            lib_pkg.dtsph_create(p)
        assert e.value.code == code, over
    # a batch's instances all reuse lists (each its own skin) or none does
    good = [lib_pkg.make_params(dict(base, graph=2, list_skin=0.01)), lib_pkg.make_params(dict(base, graph=2))]
    with pytest.raises(lib_pkg.DtsphError) as e:
        lib_pkg.dtsph_batch_create(good)
    assert e.value.code == -1


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's field offsets and
    sizes, as a C compiler lays them out (gcc on include/dtsph.h)."""
    import subprocess
    structs = {"dtsph_params": lib_pkg.dtsph_params, "dtsph_step_stats": lib_pkg.dtsph_step_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dtsph.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built CUDA library the product path raises; there is no CPU
    fallback."""
    monkeypatch.setattr(lib_pkg, "LIB_PATH", os.path.join(ROOT, "_build_missing", "libdtsph.so"))
    monkeypatch.setattr(lib_pkg, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        lib_pkg.lib()
    cfg = dict(dim=2, h=0.1, m=0.01, nu=0.01, dt=0.01)
    with pytest.raises(ImportError):
        lib_pkg.Simulation(cfg)


def test_product_package_does_not_load_the_oracle():
    """The package and its binding import nothing from oracle/ (test
    infrastructure only)."""
    import subprocess
    import sys
    code = "import sys, paper_1904_00861_gb300; assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules)"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr


def test_oracle_and_library_share_no_code():
    """The oracle includes only system headers, and no library source includes or
    imports anything from oracle/."""
    import glob
    src = open(os.path.join(ROOT, "oracle", "dtsph_oracle.c")).read()
    for inc in re.findall(r'#include\s*(\S+)', src):
        assert inc.startswith("<"), inc
    lib_files = glob.glob(os.path.join(ROOT, "paper_1904_00861_gb300", "**", "*.*"), recursive=True)
    lib_files = [f for f in lib_files if f.endswith((".cu", ".cuh", ".h", ".py")) and "_build" not in f]
    assert lib_files
    for f in lib_files:
        for line in open(f).read().splitlines():
            s = line.strip()
            if s.startswith(("#include", "import ", "from ")):
                assert "oracle" not in s, (f, s)
