"""CPU-side checks of the C ABI: the library builds, loads, and exports every function that
include/hmc.h declares; the Python binding's structs match the header's field order."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hmc.h")


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(\w+)\(", text, flags=re.M)))


def header_struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text)
    body = m.group(1)
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[\w+\]", "", decl).strip()
        if not decl:
            continue
        parts = decl.split(",")
        fields.append(parts[0].split()[-1].lstrip("*"))
        fields += [q.strip().lstrip("*") for q in parts[1:]]
    return fields


@pytest.fixture(scope="module")
def libpath():
    from paper_2204_14241_gb300 import hmc
    if not os.path.exists(hmc.LIB_PATH):
        from paper_2204_14241_gb300 import build
        build.build()
    return hmc.LIB_PATH


def test_library_exports_every_header_function(libpath):
    from paper_2204_14241_gb300 import hmc
    lib = ctypes.CDLL(libpath)
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hmc.EXPORTS)


def test_binding_struct_layouts_match_header():
    from paper_2204_14241_gb300 import hmc
    for cname, pyt in [("hmc_params", hmc.Params), ("hmc_chain", hmc.Chain), ("hmc_cg_stats", hmc.CgStats),
                       ("hmc_traj_in", hmc.TrajIn), ("hmc_traj_out", hmc.TrajOut),
                       ("hmc_traj_stats", hmc.TrajStats)]:
        assert header_struct_fields(cname) == [f[0] for f in pyt._fields_], cname


def test_binding_loads_library(libpath):
    from paper_2204_14241_gb300 import hmc
    L = hmc.lib()
    assert L.hmc_last_error(None) is not None or True
