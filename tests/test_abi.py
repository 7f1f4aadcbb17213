"""Host-side checks of the C ABI: the library builds, loads, exports every
function include/cosim.h declares, and rejects bad descriptors before any
CUDA call (so these run without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from paper_2603_07038_b300 import build as B
from paper_2603_07038_b300 import cosim as api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return api.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cosim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cosim_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(api.EXPORTED) <= set(names)


def test_binding_struct_layouts_match_header(tmp_path):
    """sizes and field offsets of the ctypes mirrors == what gcc gives the header"""
    structs = {"cosim_material": api.cosim_material, "cosim_grid_desc": api.cosim_grid_desc,
               "cosim_source": api.cosim_source, "cosim_allocator": api.cosim_allocator,
               "cosim_options": api.cosim_options, "cosim_stress_opts": api.cosim_stress_opts,
               "cosim_stress_report": api.cosim_stress_report, "cosim_peak_report": api.cosim_peak_report}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cosim.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def _create_status(p, **kw):
    h = C.c_void_p()
    desc = api.Desc(p)
    for k, v in kw.items():
        setattr(desc.c, k, v)
    o = api.cosim_options()
    o.precision = api.COSIM_FP32
    st = api.load().cosim_create(C.byref(desc.c), C.byref(o), C.byref(h))
    return st, api.cosim_last_error(None)


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 0, "grid sizes"),
    ("nmat", 0, "nmat"),
    ("cpml_cells", 40, "cpml_cells"),
])
def test_invalid_descriptor_rejected_before_cuda(lib, field, value, needle):
    p = W.tiny_package()
    st, msg = _create_status(p, **{field: value})
    assert st == api.COSIM_ERR_INVALID and needle in msg


def test_invalid_material_id_rejected(lib):
    p = W.tiny_package()
    p.mat[3, 4, 5] = 7
    st, msg = _create_status(p)
    assert st == api.COSIM_ERR_INVALID and "material id" in msg


def test_thin_cpml_axis_rejected(lib):
    p = W.uniform_box(10, 40, 40, em_bc=(2, 2, 0, 0, 0, 0), cpml_cells=8)
    st, msg = _create_status(p)
    assert st == api.COSIM_ERR_INVALID and "CPML faces x cpml_cells" in msg
    # one CPML face needs only cpml_cells + 2 cells: validation passes and creation
    # proceeds to the device (not exercised here without a GPU)


def test_null_handle_calls_are_invalid(lib):
    assert lib.cosim_em_steps(None, 1, 0) == api.COSIM_ERR_INVALID
    assert lib.cosim_thermal_steps(None, 1, 0.0) == api.COSIM_ERR_INVALID
    v = C.c_double()
    assert lib.cosim_query(None, 0, C.byref(v)) == api.COSIM_ERR_INVALID
    assert lib.cosim_read_fields_async(None, 0, 0, None, 0, 0) == api.COSIM_ERR_INVALID
    assert lib.cosim_wait_reads(None) == api.COSIM_ERR_INVALID
    lib.cosim_destroy(None)


def test_noalloc_sum_wrapper_rejects_bad_tensors_before_the_call():
    """the wrapper refuses, on the host, every tensor the kernel would read out
    of bounds (wrong dtype, strided view, n past the end) or on the wrong
    device, before it touches the library"""
    import torch
    with pytest.raises(TypeError):
        api.cosim_sum_f64_noalloc(torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError):
        api.cosim_sum_f64_noalloc(torch.zeros(8, 2, dtype=torch.float64)[:, 0])
    with pytest.raises(ValueError):
        api.cosim_sum_f64_noalloc(torch.zeros(8, dtype=torch.float64), n=9)
    with pytest.raises(ValueError):
        api.cosim_sum_f64_noalloc(torch.zeros(8, dtype=torch.float64), n=-1)
    with pytest.raises(ValueError):  # a host tensor
        api.cosim_sum_f64_noalloc(torch.zeros(8, dtype=torch.float64))
