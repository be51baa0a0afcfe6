"""The ctypes mirrors of the C ABI's structs (paper_2101_05917_gb300/_native.py)
declare the same fields, in the same order, with the same types and array lengths,
as include/diffpd.h: a field added to one side only would shift every later field
across the boundary.  Parses the header's struct declarations (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2101_05917_gb300 import _native as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "diffpd.h")

SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
           "pd_status": ctypes.c_int32}
MIRRORS = {"pd_mesh_desc": N.MeshDesc, "pd_tet_mesh_desc": N.TetMeshDesc, "pd_mesh_info": N.MeshInfo, "pd_factor_opts": N.FactorOpts,
           "pd_solver_opts": N.SolverOpts, "pd_stats": N.Stats, "pd_request": N.Request, "pd_result": N.Result}


def _header_structs():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.replace("const ", " ").split())
            if not decl:
                continue
            m = re.match(r"(\w+)\s*(.*)", decl)
            base, rest = m.group(1), m.group(2)
            for item in rest.split(","):
                item = item.strip()
                ptr = item.count("*")
                item = item.replace("*", "").strip()
                arr = re.match(r"(\w+)\s*\[(\d+)\]", item)
                fname, n = (arr.group(1), int(arr.group(2))) if arr else (item, None)
                fields.append((fname, base, ptr, n))
        out[name] = fields
    return out


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_ctypes_mirror_matches_header(cname):
    fields = _header_structs()[cname]
    mirror = MIRRORS[cname]._fields_
    assert [f[0] for f in fields] == [m[0] for m in mirror]
    for (fname, base, ptr, n), (_, ctype) in zip(fields, mirror):
        if ptr:
            assert issubclass(ctype, (ctypes._Pointer, ctypes.c_void_p)), fname
        elif n is not None:
            assert issubclass(ctype, ctypes.Array) and ctype._length_ == n and ctype._type_ is SCALARS[base], fname
        elif base in SCALARS:
            assert ctype is SCALARS[base], fname
        else:
            assert ctype is MIRRORS[base], fname
