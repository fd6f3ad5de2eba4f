"""Static checks of the CUDA sources (no GPU): every translation unit that
compiles the element kernel has its own constant bank for the derivative
tables, so each must define an upload routine and mesh setup must call it;
a unit that is missed computes with D = 0."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_12477_gb300", "csrc")


def test_every_element_kernel_unit_uploads_its_tables():
    setup = open(os.path.join(CSRC, "hb_setup.cu")).read()
    units = [f for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")
             and '#include "hb_ax2.cuh"' in open(os.path.join(CSRC, f)).read()]
    assert len(units) >= 4
    for f in units:
        text = open(os.path.join(CSRC, f)).read()
        m = re.search(r"hb_status\s+(\w+)\s*\(const double \*D_all\)\s*\{\s*return hb2::upload_tables", text)
        assert m, f"{f} defines no table upload"
        assert m.group(1) + "(D64.data())" in setup, f"{m.group(1)} is not called at setup"
