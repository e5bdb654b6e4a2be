"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/w1.h (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(w1_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1810_00118_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (w1_\w+)", out))
    assert names <= exported


def test_host_only_entry_points_work_without_gpu():
    from paper_1810_00118_gb300 import w1
    o = w1.default_options()
    assert o.check_every == 0 and o.theta == 0.5 and o.alpha == -1.0 and o.algorithm == 3
    assert w1.status_string(w1.ERR_MASS).startswith("mass")
    assert w1.status_string(99) == "unknown status"


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/w1.h, printed by a C program
    that gcc compiles against the header (no GPU needed)."""
    import subprocess
    import tempfile
    body = "\n".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = (f'#include <stdio.h>\n#include <stddef.h>\n#include "w1.h"\n'
           f'int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


def test_binding_struct_layout_matches_header():
    """ctypes mirrors of w1_options / w1_stats / w1_server_config have the C
    sizes and field offsets (taken from the header by a C compiler)."""
    from paper_1810_00118_gb300 import w1
    for struct, py in (("w1_options", w1.Options), ("w1_stats", w1._Stats), ("w1_server_config", w1.ServerConfig),
                       ("w1_level_choice", w1.LevelChoice)):
        names = [n for n, _ in py._fields_]
        got = _c_layout(struct, names)
        assert ctypes.sizeof(py) == got[0], struct
        for n, off in zip(names, got[1:]):
            assert getattr(py, n).offset == off, (struct, n)


def test_oracle_is_not_imported_by_the_product():
    """The product package never loads the oracle (the oracle is test-only)."""
    pkg = os.path.join(ROOT, "paper_1810_00118_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "w1_oracle" not in text, f


def test_ctypes_mirrors_match_the_c_layouts(tmp_path):
    """Sizes and field offsets of every struct the binding mirrors, as the C
    compiler lays them out from include/w1.h (gcc, host only)."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_1810_00118_gb300 import w1
    mirrors = {"w1_options": w1.Options, "w1_stats": w1._Stats, "w1_level_choice": w1.LevelChoice,
               "w1_server_config": w1.ServerConfig, "w1_server_info": w1.ServerInfo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "w1.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in mirrors.items():
        assert c[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert c[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_no_cpu_fallback_errors_are_loud():
    """Without a GPU, building a plan or a server fails with a W1Error (there is
    no CPU path); host tensors are refused before any call."""
    import numpy as np
    import torch
    from paper_1810_00118_gb300 import w1
    cpu = torch.zeros((8, 8, 8), dtype=torch.float32)
    with pytest.raises(TypeError):
        w1.solve3d(cpu, cpu)
    with pytest.raises(TypeError):
        w1.cp_steps(*(torch.zeros((8, 8)) for _ in range(4)), 0.125, 1, 0.01, 0.01, 4)
    with pytest.raises(TypeError):
        w1.cp_steps(np.zeros((8, 8), np.float32), *(torch.zeros((8, 8)) for _ in range(3)), 0.125, 1, 0.01, 0.01, 4)
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the no-GPU errors cannot be observed here")
    with pytest.raises(w1.W1Error):
        w1.Plan(64, 64)
    with pytest.raises(w1.W1Error):
        w1.Server(max_slots=2)
