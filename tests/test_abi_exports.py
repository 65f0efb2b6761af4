"""The C ABI: every function declared in include/*.h is exported by the library
(and nothing else of the library's internals leaks); the library loads and its
defaults are readable without a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2604_10089_gb300", "liblcp_gb300.so")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:LCP_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2604_10089_gb300.build import build
    build()
    return LIB


def test_every_declared_function_is_exported(built):
    declared = declared_functions()
    assert len(declared) >= 30, sorted(declared)
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared - exported
    assert not missing, sorted(missing)
    internal = {s for s in exported if s.startswith("_Z")}
    assert not internal, sorted(internal)[:10]


def test_library_loads_and_binding_matches(built):
    from paper_2604_10089_gb300 import _abi
    import paper_2604_10089_gb300 as L
    lib = _abi.load()
    for name in declared_functions():
        assert hasattr(lib, name)
        assert name in _abi.PROTOTYPES, name
    cfg = L.lcp_default_config()
    assert cfg.n_theta == 9 and cfg.n_phi == 18 and cfg.gmres_tol == 1e-12
    assert cfg.residual_precision == L.LCP_DF64 and cfg.precondition == 1


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs: same fields, offsets and sizes
    as the C compiler lays them out (a C program built against include/*.h)."""
    from paper_2604_10089_gb300 import _abi
    structs = [("lcp_config", _abi.lcp_config), ("lcp_stats", _abi.lcp_stats), ("lcp_contact", _abi.lcp_contact)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lcp_gb300.h"', "int main(void) {"]
    for cname, py in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_layout = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        c_layout[(name, field)] = int(value)
    for cname, py in structs:
        assert c_layout[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert c_layout[(cname, field)] == getattr(py, field).offset, (cname, field)
    # equal sizes and offsets: no header field is missing from the mirror, at the end or between


def test_footprint_estimate_counts_the_optional_buffers():
    """Host-only: the admission estimate grows by exactly the buffers each option adds (the
    self-interaction correction in FP32 and FP64, the carried forces and their pairs, the
    kept solve pairs for projected starts)."""
    import paper_2604_10089_gb300 as L
    M, nt, nph = 20, 7, 14
    ns, pairs = nt * nph, M * (M - 1) // 2
    base = dict(n_theta=nt, n_phi=nph, self_quadrature=0, warm_start=0, recycle=0, precondition=1)

    def est(**kw):
        cfg = L.lcp_default_config(**{**base, **kw})
        return L.lcp_footprint_estimate(cfg, M, 6 * M)

    b0 = est()

    def grows_by(added, **kw):   # the estimate keeps a 1/16 margin on top of the buffers
        return abs((est(**kw) - b0) - (added + added // 16)) <= 2

    assert grows_by(12 * 9 * ns * ns, self_quadrature=1)        # FP32 + FP64 copies of C
    assert grows_by(24 * pairs, warm_start=L.LCP_WARM_FORCES)    # x, start, i, j per body pair
    assert est(warm_start=L.LCP_WARM_SLIP) == b0                 # the slip start needs no extra buffer
    L3 = 3 * M * ns
    assert grows_by(8 * (L3 * 10 + 12), recycle=4)                # 2 x 4 pairs + 2 vectors + coefficients
