"""The C-ABI library builds, loads and exports every declared entry point;
struct layouts agree between the header and the binding; host-side argument
validation (no GPU work)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dd_inpaint.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_03946_gb300 import binding
    return binding.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[\w\s\*]+?\b(dd_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    from paper_2110_03946_gb300 import binding
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_struct_layout_matches_header(tmp_path):
    from paper_2110_03946_gb300 import binding as B
    probe = tmp_path / "probe.c"
    fields_p = [f for f, _ in B.dd_params._fields_]
    fields_s = [f for f, _ in B.dd_stats._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(dd_params), sizeof(dd_stats));']
    lines += [f'printf("%zu\\n", offsetof(dd_params, {f}));' for f in fields_p]
    lines += [f'printf("%zu\\n", offsetof(dd_stats, {f}));' for f in fields_s]
    lines += ["return 0;}"]
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-o", str(exe), str(probe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    vals = list(map(int, out))
    assert vals[0] == ctypes.sizeof(B.dd_params)
    assert vals[1] == ctypes.sizeof(B.dd_stats)
    offs = vals[2:]
    py = [getattr(B.dd_params, f).offset for f in fields_p] + [getattr(B.dd_stats, f).offset for f in fields_s]
    assert offs == py


def test_defaults_and_strings(lib):
    from paper_2110_03946_gb300 import binding as B
    p = B.dd_params_default()
    assert (p.block, p.overlap, p.levels) == (32, 6, 3)
    assert p.local_cg_iters >= 1 and p.max_sweeps > 0
    assert B.dd_strerror(B.DD_EEMPTYMASK).startswith("empty mask")
    assert B.dd_strerror(12345) == "unknown error"


@pytest.mark.parametrize("field,value", [("block", 24), ("overlap", 32), ("overlap", -1), ("levels", 0),
                                         ("levels", 9), ("precision", 7), ("local_cg_iters", 0),
                                         ("ml_mode", 5), ("inner_tol", 1.5), ("coarse_factor", 3),
                                         ("coarse_factor", 16), ("test_stall_polls", -1),
                                         ("correction_trigger", 1.0), ("correction_trigger", -0.1),
                                         ("final_local_rtol", 1.0), ("final_local_rtol", -0.5),
                                         ("local_atol", -1.0), ("local_atol", 1.0), ("correction_cg", -1)])
def test_invalid_params_rejected_on_host(lib, field, value):
    from paper_2110_03946_gb300 import binding as B
    p = B.dd_params_default()
    setattr(p, field, value)
    m = np.ones((8, 8), dtype=np.uint8)
    v = np.zeros((1, 8, 8), dtype=np.float32)
    rc, h = B.dd_inpaint_create(8, 8, 1, m.ctypes.data, v.ctypes.data, p)
    assert rc == B.DD_EINVAL and not h.value


def test_empty_mask_and_bad_sizes_rejected_on_host(lib):
    from paper_2110_03946_gb300 import binding as B
    p = B.dd_params_default()
    m = np.zeros((8, 8), dtype=np.uint8)
    v = np.zeros((1, 8, 8), dtype=np.float32)
    rc, h = B.dd_inpaint_create(8, 8, 1, m.ctypes.data, v.ctypes.data, p)
    assert rc == B.DD_EEMPTYMASK and not h.value
    m[3, 3] = 1
    for H, W, C in [(0, 8, 1), (8, -1, 1), (8, 8, 0)]:
        rc, h = B.dd_inpaint_create(H, W, C, m.ctypes.data, v.ctypes.data, p)
        assert rc == B.DD_EINVAL
    rc, h = B.dd_inpaint_create(8, 8, 1, None, v.ctypes.data, p)
    assert rc == B.DD_EINVAL
    assert B.dd_inpaint_destroy(None) == B.DD_OK
    assert B.dd_inpaint_solve(None, 0, 1e-6) == B.DD_EINVAL


def test_library_has_no_cpu_fallback_symbols(lib):
    """The product path has no host compute entry: the only exported names
    are the declared dd_* entry points."""
    out = subprocess.check_output(["nm", "-D", "--defined-only",
                                   os.path.join(ROOT, "paper_2110_03946_gb300", "libdd_inpaint.so")]).decode()
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("dd_")})
    assert exported == _declared()


def test_device_budget_accounting_without_handles(lib):
    # no handle is alive in this process on the CPU: nothing is held, and the
    # budget setter takes any value (0 restores "no cap")
    from paper_2110_03946_gb300 import binding as B
    assert B.dd_device_bytes_in_use() == 0
    B.dd_set_device_budget(1 << 20)
    B.dd_set_device_budget(0)
    assert B.dd_device_bytes_in_use() == 0


def test_fma_peak_rejects_bad_arguments(lib):
    import ctypes as ct
    from paper_2110_03946_gb300 import binding as B
    t = ct.c_double(0.0)
    assert lib.dd_fp32_fma_peak(0, ct.byref(t), None, None) == B.DD_EINVAL
    assert lib.dd_fp32_fma_peak(3, None, None, None) == B.DD_EINVAL
