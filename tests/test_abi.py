"""C-ABI checks that need no GPU: the library loads, exports every entry point declared in
include/mb.h, validates descriptors on the host, and reports injected allocation failures."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mb.h")).read()
    return sorted(set(re.findall(r"^(?:mb_status|const char\*)\s+(mb_\w+)\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mb_create_grid", "mb_destroy", "mb_set_particles", "mb_step",
              "mb_get_velocities", "mb_spread", "mb_interp", "mb_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1407_5600_gb300 as mb
    lib = mb.load_library()
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", mb._LIB_PATH], capture_output=True,
                         text=True).stdout
    for n in _declared():
        assert re.search(r" T " + n + r"$", out, re.M), n


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 3, "powers of two"), ("ny", 512, "powers of two"), ("batch", 0, "batch"),
    ("h", 0.0, "positive"), ("eta", -1.0, "positive"), ("precision", 2, "precision"),
    ("advection", 2, "advection"), ("kT", -1e-3, "kT"), ("kT", float("nan"), "kT"),
    ("mean_mode", 3, "mean_mode"), ("integrator", 2, "integrator"),
])
def test_descriptor_validation_is_host_side(field, value, msg):
    import paper_1407_5600_gb300 as mb
    d = mb.GridDesc(16, 16, 16)
    setattr(d, field, value)
    with pytest.raises(mb.MBError) as ei:
        mb.create_grid(d)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_injected_allocation_failure_reports_enomem():
    code = ("import paper_1407_5600_gb300 as mb\n"
            "try:\n    mb.create_grid(mb.GridDesc(8, 8, 8))\n"
            "except mb.MBError as e:\n    print('STATUS', e.status, e)\n")
    env = dict(os.environ, MB_FAULT_ALLOC="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         cwd=ROOT, timeout=120).stdout
    assert "STATUS 2" in out and "injected allocation failure" in out
