"""C-ABI library: builds, loads without a GPU, exports every declared symbol; host-side
tree validation rejects malformed trees (CPU only)."""
import os
import re
import shutil

import numpy as np
import pytest

from paper_2603_23891_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    out = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        out |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fgs_\w+)\s*\(", txt, flags=re.M))
    return out


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2603_23891_gb300 import build
    build.build()
    from paper_2603_23891_gb300 import filtergs
    return filtergs


def test_exports_every_declared_symbol(lib):
    L = lib.lib()
    declared = _declared_symbols()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L, name), name
    assert set(lib.EXPORTED) == declared
    assert L.fgs_version() == 3


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(lib.FgsError):
        lib.fgs_create(0)


def _mutated(tree, **changes):
    import copy
    t = copy.copy(tree)
    for k, v in changes.items():
        setattr(t, k, v)
    return t


def test_validate_tree(lib):
    tree = synth.random_small_tree(0, n_leaves=120, branching=(2, 5), sh_degree=1)
    code, msg = lib.fgs_validate_tree(tree)
    assert code == lib.FGS_OK, msg

    par = tree.parent.copy()
    par[5] = 5                                             # self loop
    assert lib.fgs_validate_tree(_mutated(tree, parent=par))[0] == lib.FGS_ERR_TREE
    par = tree.parent.copy()
    par[7] = tree.n + 3                                     # out of range
    assert lib.fgs_validate_tree(_mutated(tree, parent=par))[0] == lib.FGS_ERR_TREE
    par = tree.parent.copy()
    par[3] = -1                                             # two roots
    assert lib.fgs_validate_tree(_mutated(tree, parent=par))[0] == lib.FGS_ERR_TREE
    # cycle: root's child points to a grandchild
    par = tree.parent.copy()
    kid = int(np.nonzero(par == 0)[0][0])
    grand = int(np.nonzero(par == kid)[0][0])
    par[kid] = grand
    assert lib.fgs_validate_tree(_mutated(tree, parent=par))[0] == lib.FGS_ERR_TREE
    ap = tree.ap.copy()
    ap[0, 10] = (ap[0, 10] + 1) % tree.n                    # AP disagrees with parent
    assert lib.fgs_validate_tree(_mutated(tree, ap=ap))[0] == lib.FGS_ERR_TREE
    ap = tree.ap[:-1].copy()                                # depth too small
    assert lib.fgs_validate_tree(_mutated(tree, ap=ap))[0] == lib.FGS_ERR_TREE
    leaf = tree.is_leaf.copy()
    leaf[0] = 1                                             # root marked leaf
    assert lib.fgs_validate_tree(_mutated(tree, is_leaf=leaf))[0] == lib.FGS_ERR_TREE
    mu = tree.mu.copy()
    mu[1, 4] = np.nan
    assert lib.fgs_validate_tree(_mutated(tree, mu=mu))[0] == lib.FGS_ERR_TREE
    op = tree.opacity.copy()
    op[2] = 0.0
    assert lib.fgs_validate_tree(_mutated(tree, opacity=op))[0] == lib.FGS_ERR_TREE
    sh = tree.sh.copy()
    sh[3, 1, 2] = np.inf
    assert lib.fgs_validate_tree(_mutated(tree, sh=sh))[0] == lib.FGS_ERR_TREE


_STRUCTS = ["fgs_tree", "fgs_camera", "fgs_params", "fgs_stats", "fgs_gauss_params", "fgs_gauss_grads"]


def test_binding_layouts_match_the_header(tmp_path):
    """Every struct the ctypes binding passes has the header's size and field offsets (a C
    program compiled against include/filtergs.h prints them), and every FGS_* integer
    constant the binding defines has the header's value."""
    import ctypes
    import subprocess
    from paper_2603_23891_gb300 import filtergs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "filtergs.h"', "int main(void) {"]
    for s in _STRUCTS:
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(filtergs, s)._fields_:
            lines.append(f'printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for s in _STRUCTS:
        cls = getattr(filtergs, s)
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert got[(s, name)] == getattr(cls, name).offset, (s, name)
    header = open(os.path.join(ROOT, "include", "filtergs.h")).read()
    consts = {m.group(1): int(m.group(2).rstrip("u"), 0)
              for m in re.finditer(r"^#define (FGS_\w+) \(?(-?\w+)\)?", header, flags=re.M)
              if re.fullmatch(r"-?(0x[0-9a-fA-F]+|\d+)u?", m.group(2))}
    checked = 0
    for name, v in consts.items():
        if hasattr(filtergs, name):
            assert getattr(filtergs, name) == v, name
            checked += 1
    assert checked >= 10


def test_null_arguments_rejected_before_any_cuda_call(lib):
    """Every entry point checks its context and output pointers before it touches the
    GPU: with a null context (or null buffers) each returns FGS_ERR_ARG, here on a
    machine without a GPU; fgs_destroy(NULL) is a no-op, fgs_last_error(NULL) a fixed
    string, and the context-free entry points reject bad sizes before any launch."""
    import ctypes
    L = lib.lib()
    special = {"fgs_version", "fgs_destroy", "fgs_last_error", "fgs_validate_tree", "fgs_eval_exp",
               "fgs_compact_selection_noalloc"}
    checked = 0
    for name in lib.EXPORTED:
        if name in special:
            continue
        f = getattr(L, name)
        args = [0.0 if t is ctypes.c_float else 0 if t in (ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                                          ctypes.c_size_t) else None
                for t in f.argtypes]
        assert f(*args) == lib.FGS_ERR_ARG, name
        checked += 1
    assert checked == len(lib.EXPORTED) - len(special)
    assert L.fgs_destroy(None) == lib.FGS_OK
    assert L.fgs_last_error(None) == b"null context"
    msg = ctypes.create_string_buffer(128)
    assert L.fgs_validate_tree(None, msg, 128) == lib.FGS_ERR_ARG and msg.value == b"null tree"
    assert L.fgs_eval_exp(None, None, 0, None) == lib.FGS_OK          # nothing to do
    assert L.fgs_eval_exp(None, None, 5, None) == lib.FGS_ERR_ARG
    nz = ctypes.c_void_p(0x1000)                                         # never dereferenced
    noalloc = L.fgs_compact_selection_noalloc
    assert noalloc(None, 4, nz, nz, None) == lib.FGS_ERR_ARG
    assert noalloc(nz, 0, nz, nz, None) == lib.FGS_ERR_ARG
    assert noalloc(nz, (1 << 26) + 1, nz, nz, None) == lib.FGS_ERR_ARG   # above the scratch's limit
