"""Every call of the boundary that carries a step of the method names the
passage of the paper that defines it in its comment in include/colatus.h
(an equation, a section or the appendix), beside argument meaning, layout,
ownership and errors.  No GPU is needed."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "colatus.h")).read()
CITE = re.compile(r"(Eqs?\.\s*\d|Sec\.\s*[IVX]+|Appendix\s*[A-Z])")

CALLS = ["colatus_init", "colatus_set_config", "colatus_set_state", "colatus_get_state", "colatus_forces",
         "colatus_step", "colatus_record_tracers", "colatus_read_tracers", "colatus_diagnostics",
         "colatus_force_vjp", "colatus_adjoint_forward", "colatus_adjoint_backward", "colatus_tangent_init",
         "colatus_tangent_step", "colatus_set_periodic", "colatus_set_deformation", "colatus_velocity_spectrum",
         "colatus_tracer_spectrum", "colatus_ensemble_init", "colatus_ensemble_forces", "colatus_ensemble_step",
         "colatus_selftest_sym_tables"]


def comment_before(name):
    """The comment block that ends closest above the declaration of `name`."""
    decl = re.search(r"^[a-z][\w \*]*\b" + name + r"\(", HEADER, re.M)
    assert decl, name
    end = HEADER.rfind("*/", 0, decl.start())
    start = HEADER.rfind("/*", 0, end)
    assert 0 <= start < end, name
    between = HEADER[end + 2:decl.start()]
    # only other declarations (of the same group) may sit between the comment and this one
    assert "/*" not in between, name
    return HEADER[start:end]


@pytest.mark.parametrize("name", CALLS)
def test_call_cites_its_passage(name):
    assert CITE.search(comment_before(name)), name
