"""Host-only checks of the C ABI: the library builds, loads, exports every symbol
declared in include/pdcs.h, and its argument validation (which runs before any
CUDA call) rejects bad input with PDCS_ERR_INVALID."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import pdcs as P
from paper_2505_00311_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pdcs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdcs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "pdcs_create" in names and "pdcs_solve" in names and "pdcs_get_solution" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in P.SIGNATURES, name


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a probe against include/pdcs.h with gcc and compare sizes and offsets."""
    import subprocess
    structs = {"pdcs_csr": P.pdcs_csr, "pdcs_cone": P.pdcs_cone, "pdcs_options": P.pdcs_options,
               "pdcs_info": P.pdcs_info, "pdcs_state": P.pdcs_state, "pdcs_state_arrays": P.pdcs_state_arrays}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdcs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)


def test_default_options(lib):
    o = P.pdcs_default_options()
    assert o.rescale == P.RESCALE_COORD and o.ruiz_iters == 10 and o.check_period == 64
    assert o.beta == 1.0 and o.step_mode == P.STEP_ADAPTIVE and o.use_graphs == 1


def _bad(prob, **opts):
    with pytest.raises(P.PdcsError) as e:
        P.pdcs_create(prob, P.pdcs_default_options(**opts))
    assert e.value.status == P.ERR_INVALID
    return str(e.value)


def test_validation_rejects_bad_input(lib):
    p = I.small_socp(0, n=40, m=20, row_nnz=4, n_nonneg=10, n_soc=1, soc_dim=10)
    q = dict(p); q["col"] = p["col"].copy(); q["col"][3] = 40
    assert "column" in _bad(q)
    q = dict(p); q["row_ptr"] = p["row_ptr"].copy(); q["row_ptr"][5], q["row_ptr"][6] = q["row_ptr"][6], q["row_ptr"][5]
    _bad(q)
    q = dict(p); q["cone_dims"] = np.array([10, 9])
    assert "sum" in _bad(q)
    q = dict(p); q["cone_types"] = np.array([P.CONE_NONNEG, 7])
    _bad(q)
    q = dict(p); q["cone_types"] = np.array([P.CONE_NONNEG, P.CONE_EXP])
    assert "dimension" in _bad(q)
    q = dict(p); q["val"] = p["val"].copy(); q["val"][0] = np.nan
    _bad(q)
    q = dict(p); q["h"] = p["h"].copy(); q["h"][0] = np.inf
    _bad(q)
    q = dict(p); q["lb"] = np.ones(40); q["ub"] = np.zeros(40)
    assert "lb > ub" in _bad(q)
    q = dict(p); q["cone_types"] = np.array([], dtype=np.int32); q["cone_dims"] = np.array([], dtype=np.int64)
    assert "empty" in _bad(q)
    _bad(p, check_period=0)
    _bad(p, beta=1.5)
    _bad(p, spmv_lanes=3)
    q = dict(p); q["m"] = 0
    _bad(q)


def test_validation_rejects_bad_primal_cones(lib):
    p = I.primal_cone_program(seed=7, n_before=6, pcone_dims=(4, 5), n_after=3, m=16, row_nnz=4)
    assert "lb = -inf" in _bad(dict(p, lb=np.zeros(p["n"])))
    assert "SOC" in _bad(dict(p, pcone_types=np.array([P.CONE_SOC, P.CONE_EXP], np.int32)))
    assert "SOC" in _bad(dict(p, pcone_types=np.array([P.CONE_SOC, P.CONE_RSOC], np.int32),
                              pcone_dims=np.array([4, 1], np.int64)))
    assert "exceed" in _bad(dict(p, pcone_start=p["n"] - 3))
    assert "FP64" in _bad(p, precision=P.PRECISION_FP32)
    assert "FP64" in _bad(p, fuse_primal=1)
    assert "FP64" in _bad(p, batch_blocks=64)


def test_missing_library_fails_loudly():
    """No CPU fallback: without the CUDA library every entry point raises."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2505_00311_gb300 import pdcs as P, instances as I\n"
            "P.LIB_PATH = '/nonexistent/libpdcs.so'\n"
            "try:\n"
            "    P.Solver(I.small_socp(0))\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "missing" in r.stdout


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_00311_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "pdcs_oracle.h" not in text and "liborc" not in text, f
