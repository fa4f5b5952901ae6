"""The C-ABI library loads and exports every entry point include/mnl.h declares.

These tests need no GPU: they only open the shared library and call the two
pure-host functions (parameter count, status text).
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mnl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(mnl_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1404_3177_gb300 import _build, _native
    _build.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mnl_create", "mnl_loglik_grad", "mnl_hessian", "mnl_newton_step", "mnl_fit", "mnl_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1404_3177_gb300 import _native
    names = declared_functions()
    assert set(names) == set(_native.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_num_params_and_status_strings(lib):
    from paper_1404_3177_gb300 import _native as nat
    assert nat.mnl_num_params(nat.mnl_dims(2000, 5, 4, 1, 2, 0)) == 22
    assert nat.mnl_num_params(nat.mnl_dims(200000, 50, 50, 5, 5, 0)) == 2700
    assert nat.mnl_num_params(nat.mnl_dims(500000, 100, 100, 0, 10, 0)) == 9910
    assert nat.mnl_num_params(nat.mnl_dims(1182, 4, 2, 1, 1, 1)) == 11  # Fish model, gamma_0 estimated
    assert nat.mnl_num_params(nat.mnl_dims(0, 5, 4, 1, 2, 0)) == -1
    assert nat.mnl_num_params(nat.mnl_dims(10, 1, 4, 1, 2, 0)) == -1
    for s in range(10):
        assert nat.mnl_status_string(s)
    assert "unknown" in nat.mnl_status_string(99)


def test_fit_opts_defaults(lib):
    from paper_1404_3177_gb300 import _native as nat
    o = nat.mnl_fit_opts_default()
    assert o.maxiter == 50 and o.max_halvings == 30 and o.gtol == 1e-8 and o.ftol == 0.0 and o.steptol < 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1404_3177_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "mnl_oracle" not in txt, fn
