"""CPU-side checks of the C-ABI library: it loads, exports every declared
symbol, and its host-only logic (interface detection, DD order, input
validation, SPD detection) is exact.  No GPU compute is called here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import slrgen
from oracle.slr_oracle import dd_order as oracle_dd_order

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_04340_gb300 import slr
    return slr.load()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "slr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(slr_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    from paper_1505_04340_gb300 import slr
    names = _declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(slr.EXPORTS) == [n for n in names if n in slr.EXPORTS]
    assert set(names) == set(slr.EXPORTS)


@pytest.mark.parametrize("dims,boxes", [((32, 32), (2, 2)), ((30, 17), (3, 2)), ((12, 11, 10), (2, 3, 2)),
                                        ((9, 9), (1, 1)), ((20, 20, 20), (4, 4, 4))])
def test_dd_order_bit_exact_vs_oracle(lib, dims, boxes):
    from paper_1505_04340_gb300 import dd_order
    rp, ci, v = slrgen.laplacian(dims)
    part = slrgen.box_partition(dims, boxes)
    p = int(np.prod(boxes))
    perm, io, fo, s = dd_order(rp, ci, part, p)
    o = oracle_dd_order(rp, ci, part, p)
    assert s == o.s
    assert np.array_equal(perm, o.perm)
    assert np.array_equal(io, o.int_off) and np.array_equal(fo, o.ifc_off)


@pytest.mark.parametrize("dims,boxes", [((32, 32), (2, 2)), ((30, 17), (3, 2)), ((12, 11, 10), (2, 3, 2))])
def test_dd_order_with_vertex_separators_vs_oracle(lib, dims, boxes):
    """part = -1 marks separator vertices: the library's order equals the oracle's, the
    separators come last, and every part's interface group is empty (the separators
    disconnect the boxes)."""
    from paper_1505_04340_gb300 import dd_order
    rp, ci, v = slrgen.laplacian(dims)
    part = slrgen.box_partition_vsep(dims, boxes)
    p = int(np.prod(boxes))
    perm, io, fo, s = dd_order(rp, ci, part, p)
    o = oracle_dd_order(rp, ci, part, p)
    assert s == o.s == int(np.sum(part < 0))
    assert np.array_equal(perm, o.perm)
    assert np.array_equal(io, o.int_off) and np.array_equal(fo, o.ifc_off) and fo[-1] == 0
    assert np.all(part[perm[len(perm) - s:]] == -1)


def test_dd_order_random_partition(lib):
    from paper_1505_04340_gb300 import dd_order
    rp, ci, v = slrgen.laplacian((15, 14))
    part = (slrgen.splitmix64(9, 15 * 14) % np.uint64(5)).astype(np.int32)
    perm, io, fo, s = dd_order(rp, ci, part, 5)
    o = oracle_dd_order(rp, ci, part, 5)
    assert np.array_equal(perm, o.perm) and s == o.s


def _setup_status(lib, rp, ci, v, part, p, fields=None):
    from paper_1505_04340_gb300 import slr
    o = slr.Opts()
    lib.slr_default_opts(C.byref(o))
    for name, r in (fields or {}).items():
        if isinstance(name, int):
            o.reserved[name] = r
        else:
            setattr(o, name, r)
    h = C.c_void_p()
    rp, ci, part = (np.ascontiguousarray(a, dtype=np.int32) for a in (rp, ci, part))
    v = np.ascontiguousarray(v, dtype=np.float64)
    st = lib.slr_setup(len(rp) - 1, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, p, part.ctypes.data,
                       C.byref(o), None, C.byref(h))
    assert not h.value
    return st


def test_setup_rejects_bad_input_before_any_device_work(lib):
    rp, ci, v = slrgen.laplacian((6, 5))
    part = slrgen.box_partition((6, 5), (2, 1))
    bad = ci.copy()
    bad[3] = 999                                     # column out of range
    assert _setup_status(lib, rp, bad, v, part, 2) == 1
    asym = v.copy()
    asym[1] += 0.5                                   # values no longer symmetric
    assert _setup_status(lib, rp, ci, asym, part, 2) == 1
    assert _setup_status(lib, rp, ci, v, part + 5, 2) == 1   # part out of range
    assert _setup_status(lib, rp, ci, v, part - 2, 2) == 1   # below -1 (the separator mark)
    assert "range" in lib.slr_last_error_message().decode()


BAD_OPTIONS = [{"band_split": 3}, {"host_loop": 2}, {"band_slots": 1}, {"band_slots": 9}, {"c_persistent": 2},
               {"autotune": -1}, {"autotune": 2}, {"target_kappa": 1}, {"target_kappa": -3}, {"band_threads": 128},
               {"band_threads": 1024}, {"c_levels_only": 2}, {"c_levels_only": -1}, {"band_factor_host": 2},
               {"indefinite": 2}, {"band_order": 4}, {"band_order": -1}, {"u_dtype": 3}, {"u_dtype": -1},
               {"u_dtype": 1},                     # a tensor-core dtype needs the mixed path
               {"spin_limit": -5}, {"band_mma": 3}, {"band_mma": 1},   # tensor cores need the mixed path
               {"zform": 2}, {"zform": -1}, {0: 1}, {5: 1}]


@pytest.mark.parametrize("fields", BAD_OPTIONS)
def test_setup_rejects_bad_tuning_options(lib, fields):
    """Execution choices, method options and the reserved tail: out-of-range values
    are refused before any device work."""
    rp, ci, v = slrgen.laplacian((6, 5))
    part = slrgen.box_partition((6, 5), (2, 1))
    assert _setup_status(lib, rp, ci, v, part, 2, fields) == 1
    assert "invalid options" in lib.slr_last_error_message().decode()


def test_opts_layout_matches_header(lib):
    """The binding's slr_opts mirrors include/slr.h field for field (names and order)."""
    import re
    from paper_1505_04340_gb300 import slr
    hdr = open(os.path.join(ROOT, "include", "slr.h")).read()
    body = hdr[hdr.index("typedef struct {", hdr.index("SLR_U_FP32")):hdr.index("} slr_opts;")]
    names = re.findall(r"^\s*(?:int32_t|uint64_t)\s+(\w+)", body, flags=re.M)
    assert names == [f for f, _ in slr.Opts._fields_]


@pytest.mark.parametrize("struct", ["slr_opts", "slr_info"])
def test_struct_offsets_match_header(struct, tmp_path):
    """Every field of the binding's slr_opts / slr_info sits at the offset the C compiler
    gives it in include/slr.h, and the sizes agree (a program built with gcc prints them)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1505_04340_gb300 import slr
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    cls = slr.Opts if struct == "slr_opts" else slr.Info
    names = [f for f, _ in cls._fields_]
    src = tmp_path / "offsets.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"slr.h\"\nint main(void) {\n" +
                   "".join(f'  printf("%zu\\n", offsetof({struct}, {n}));\n' for n in names) +
                   f'  printf("%zu\\n", sizeof({struct}));\n  return 0;\n}}\n')
    exe = tmp_path / "offsets"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [getattr(cls, n).offset for n in names] + [ctypes.sizeof(cls)]
    assert got == want, dict(zip(names + ["sizeof"], zip(got, want)))


def test_setup_detects_non_spd_block(lib):
    rp, ci, v = slrgen.laplacian((6, 5))
    v = v.copy()
    diag = np.array([q for i in range(30) for q in range(rp[i], rp[i + 1]) if ci[q] == i])
    v[diag[7]] = -4.0                                # an interior node of part 0 loses positivity
    part = slrgen.box_partition((6, 5), (2, 1))
    assert _setup_status(lib, rp, ci, v, part, 2) == 2


def test_status_strings(lib):
    assert lib.slr_status_str(0) == b"SLR_OK"
    assert lib.slr_status_str(5) == b"SLR_ERR_NOT_CONVERGED"
