"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports every
function include/rbl.h declares, and validates parameters on the host."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2105_04884_gb300 import _build, rbl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbl_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return rbl.load()


def test_exports_match_header(lib):
    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rbl_[a-z_]+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert sorted(rbl.EXPORTS) == declared
    for name in declared:
        getattr(lib, name)


def test_params_default_and_status_strings(lib):
    prm = rbl.rbl_params()
    lib.rbl_params_default(ctypes.byref(prm))
    assert prm.cells_per_cutoff == 2 and prm.subtract_net_force == 1 and prm.precision == rbl.RBL_FP32
    assert prm.p == 10 and prm.dt == 0.005 and prm.sampling == rbl.RBL_SAMPLE_SHELL
    assert prm.potential == rbl.RBL_POT_LJ and prm.alpha == 0.0 and prm.rho_cap == 0.0
    for code, name in rbl.STATUS.items():
        assert lib.rbl_status_string(code).decode() == name


def _size(prm, N):
    s = ctypes.c_size_t()
    st = rbl.load().rbl_workspace_size(ctypes.byref(prm), N, ctypes.byref(s))
    return st, s.value


def test_workspace_size_and_validation(lib):
    prm = rbl.make_params([10.772] * 3, 1.5, 3.5, 0.3, 10, 0.005)
    st, n1 = _size(prm, 1000)
    assert st == 0 and n1 > 1000 * 200
    st, n2 = _size(prm, 2000)
    assert st == 0 and n2 > n1
    bad = [
        dict(r_c=3.5, r_s=1.5),                 # r_c >= r_s
        dict(p=0), dict(p=129),                 # batch size range
        dict(dt=0.0), dict(skin=-0.1),
        dict(L=[7.0, 10.772, 10.772]),          # box below 2 (r_s + skin)
        dict(cells_per_cutoff=4),
        dict(T=float("nan")),
        dict(potential=2),                      # unknown pair potential
        dict(potential=1, alpha=0.0),           # Ewald term without a splitting parameter
        dict(potential=1, alpha=float("inf")),
    ]
    for kw in bad:
        args = dict(L=[10.772] * 3, r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005)
        args.update(kw)
        prm = rbl.make_params(**args)
        assert _size(prm, 1000)[0] == 1, kw
    assert _size(rbl.make_params([10.772] * 3, 1.5, 3.5, 0.3, 10, 0.005), 1)[0] == 1  # N < 2
    # the Ewald term adds the charge arrays to the workspace
    st, ne = _size(rbl.make_params([10.772] * 3, 1.5, 3.5, 0.3, 10, 0.005, potential=rbl.RBL_POT_LJ_EWALD,
                                   alpha=1.0), 1000)
    assert st == 0 and ne > n1


def test_create_rejects_bad_workspace(lib):
    prm = rbl.make_params([10.772] * 3, 1.5, 3.5, 0.3, 10, 0.005)
    h = ctypes.c_void_p()
    st = lib.rbl_create(ctypes.byref(prm), 1000, None, 0, None, ctypes.byref(h))
    assert st in (1, 2)
    assert b"workspace" in lib.rbl_last_error(h)
    lib.rbl_destroy(h)


def test_product_has_no_oracle_dependency():
    """The library and its binding never reach the CPU oracle."""
    for sub in ("paper_2105_04884_gb300",):
        for dirpath, _, files in os.walk(os.path.join(ROOT, sub)):
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h")):
                    text = open(os.path.join(dirpath, f)).read()
                    assert "import oracle" not in text and "from oracle" not in text, f
                    assert "rbl_oracle" not in text, f


def test_batch_validation(lib):
    """Replicas may differ in box, temperature, seed and N only."""
    def size(prms, Ns):
        arr = (rbl.rbl_params * len(prms))(*prms)
        nn = (ctypes.c_int * len(Ns))(*Ns)
        s = ctypes.c_size_t()
        return lib.rbl_workspace_size_batch(arr, len(prms), nn, ctypes.byref(s)), s.value

    a = rbl.make_params([10.772] * 3, 1.5, 3.5, 0.3, 10, 0.005, T=1.5, seed=1)
    b = rbl.make_params([12.0, 12.5, 13.0], 1.5, 3.5, 0.3, 10, 0.005, T=1.1, seed=7)
    st, n2 = size([a, b], [1000, 1500])
    assert st == 0
    st1, n1 = size([a], [1000])
    assert st1 == 0 and n2 > n1
    assert size([a, b], [1000, 1])[0] == 1                              # N < 2 in one replica
    for field, val in (("r_c", 1.2), ("p", 5), ("dt", 0.002), ("precision", rbl.RBL_FP64),
                       ("full_list", 1), ("cells_per_cutoff", 1), ("gamma", 1.0)):
        c = rbl.make_params([12.0] * 3, 1.5, 3.5, 0.3, 10, 0.005)
        setattr(c, field, val)
        assert size([a, c], [1000, 1000])[0] == 1, field
    h = ctypes.c_void_p()
    assert lib.rbl_create_batch(None, 0, None, None, 0, None, ctypes.byref(h)) == 1
    lib.rbl_destroy(h)
    assert lib.rbl_replicas(None) == 0


def test_struct_layouts_match_header(tmp_path):
    """rbl_params and rbl_obs as the C compiler lays them out from include/rbl.h equal
    the ctypes structures the binding passes (field offsets and total size)."""
    import os
    import subprocess

    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rbl.h"', "int main(void) {"]
    for st in (rbl.rbl_params, rbl.rbl_obs):
        name = st.__name__
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["cc", "-I", inc, "-o", str(exe), str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, value = line.split()
        st = rbl.rbl_params if name == "rbl_params" else rbl.rbl_obs
        expect = ctypes.sizeof(st) if field == "sizeof" else getattr(st, field).offset
        assert int(value) == expect, (name, field, value, expect)
        seen += 1
    assert seen == 2 + len(rbl.rbl_params._fields_) + len(rbl.rbl_obs._fields_)


def test_tune_cells_workspace_size(lib):
    """The cell-size tuner's workspace is the largest of the three per-K workspaces
    (whatever K the parameters carry), and invalid parameters are refused; the tuner
    itself refuses missing arrays and a step count below 1 before touching a GPU."""
    base = dict(L=[12.0, 13.0, 20.0], r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005)
    sizes = [_size(rbl.make_params(cells_per_cutoff=k, **base), 3000) for k in (1, 2, 3)]
    assert all(st == 0 for st, _ in sizes)
    for k in (1, 2, 3):
        s = ctypes.c_size_t()
        assert lib.rbl_tune_cells_workspace_size(ctypes.byref(rbl.make_params(cells_per_cutoff=k, **base)), 3000,
                                                 ctypes.byref(s)) == 0
        assert s.value == max(n for _, n in sizes)
    s = ctypes.c_size_t()
    bad = rbl.make_params(**dict(base, r_c=3.5, r_s=1.5))
    assert lib.rbl_tune_cells_workspace_size(ctypes.byref(bad), 3000, ctypes.byref(s)) == 1
    K = ctypes.c_int()
    prm = rbl.make_params(**base)
    x = np.zeros((3000, 3))
    assert lib.rbl_tune_cells(ctypes.byref(prm), 3000, None, None, None, 0, None, 10, ctypes.byref(K), None) == 1
    assert lib.rbl_tune_cells(ctypes.byref(prm), 3000, x.ctypes.data_as(ctypes.c_void_p), None,
                              ctypes.c_void_p(256), 1 << 30, None, 0, ctypes.byref(K), None) == 1
