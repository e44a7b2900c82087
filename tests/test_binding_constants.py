"""The binding's numeric constants (precisions, prd_set_option ids and their
values, error codes) equal the ones include/prd.h declares, read from the
header's enums as text: a renumbering on one side fails here, without a GPU."""
import os
import re

from paper_2505_20968_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_enums():
    text = open(os.path.join(ROOT, "include", "prd.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, v in re.findall(r"(PRD_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            vals[name] = int(v)
    return vals


def test_binding_constants_match_the_header():
    h = _header_enums()
    names = [n for n in dir(binding) if n.startswith("PRD_") and isinstance(getattr(binding, n), int)]
    assert len(names) >= 15
    for n in names:
        if n == "PRD_OK":
            continue
        assert n in h, f"{n} is not declared in include/prd.h"
        assert getattr(binding, n) == h[n], (n, getattr(binding, n), h[n])
    for code, name in binding.ERRORS.items():
        assert h[name] == code, (name, code, h[name])
    # every option the header declares has a binding constant
    for n in h:
        if n.startswith("PRD_OPT_"):
            assert hasattr(binding, n), n
