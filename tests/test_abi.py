"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/vd.h (no compute call: no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vd_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2509_07175_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2509_07175_b300 import binding
    assert sorted(binding.exported_symbols()) == _declared()


def test_strerror_without_gpu():
    from paper_2509_07175_b300 import binding, build
    build.build()
    lib = binding.load()
    assert lib.vd_strerror(-4) == b"capacity exceeded (polytope, queue, pair set or flag buffer)"
    assert lib.vd_strerror(0) == b"ok"
    assert lib.vd_strerror(-9) == b"two sites coincide"
    # every error code of the header has a name
    src = open(os.path.join(ROOT, "include", "vd.h")).read()
    for code in re.findall(r"VD_ERR_[A-Z]+ = (-\d+)", src):
        assert lib.vd_strerror(int(code)) != b"unknown error", code


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2509_07175_b300 import binding, build
    build.build()
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.vd_create(ctypes.byref(h), None, 10, 3, 0) == -1
    assert lib.vd_create(ctypes.byref(h), ctypes.c_void_p(16), 0, 3, 0) == -1
    assert lib.vd_create(ctypes.byref(h), ctypes.c_void_p(16), 10, 4, 0) == -1
    assert lib.vd_create(ctypes.byref(h), ctypes.c_void_p(16), 10, 3, 7) == -1


def _c_layout(struct, fields, tmp_path):
    """sizeof and field offsets of a struct of include/vd.h, from gcc."""
    import subprocess
    src = tmp_path / f"layout_{struct}.c"
    body = "".join(f'  printf("%s %zu\\n", "{f}", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text(f'#include <stddef.h>\n#include <stdio.h>\n#include "vd.h"\nint main(void) {{\n'
                   f'  printf("sizeof %zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / f"layout_{struct}"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split()
    return {k: int(v) for k, v in zip(out[::2], out[1::2])}


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes mirrors of vd_options, vd_result and vd_pieces have the C layout:
    the same size and the same offset for every field (a field added on one side
    only would shift the others silently)."""
    from paper_2509_07175_b300 import binding as B
    for struct, cls in (("vd_options", B.Options), ("vd_result", B.Result), ("vd_pieces", B.PiecesC)):
        names = [f[0] for f in cls._fields_]
        c = _c_layout(struct, names, tmp_path)
        assert c["sizeof"] == ctypes.sizeof(cls), struct
        for name in names:
            assert c[name] == getattr(cls, name).offset, (struct, name)
