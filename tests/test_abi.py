"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU, exports every
function include/cpic.h declares, and the binding declares the same set (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(HEADER):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(cpic_[a-z_0-9]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1311_2286_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["cpic_create", "cpic_destroy", "cpic_set_map_vertices", "cpic_load_particles", "cpic_step",
              "cpic_push", "cpic_solve_field", "cpic_get_diag", "cpic_sort", "cpic_inject"]:
        assert n in names
    assert len(names) >= 25


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_without_gpu_and_binding_matches(lib_path):
    from paper_1311_2286_gb300 import cpic

    lib = cpic.load(lib_path)
    assert lib.cpic_abi_version() == 1
    assert set(cpic.exported_symbols()) == declared_functions()
    assert lib.cpic_status_string(-4) == b"field solve did not converge"


def test_footprint_and_validation_are_host_only(lib_path):
    from paper_1311_2286_gb300 import cpic

    cpic.load(lib_path)
    cfg = cpic.make_config(2, (128, 256), [1, 1, 0, 0], [-5, 0, 0, 0], [1, 1, 0, 0], 0.1,
                           [(-1, 1, 1e-3, 3_000_000), (1, 1836, 1e-3, 3_000_000)])
    nbytes = cpic.Run.footprint(cfg)
    # two particle buffers of 24 B per slot dominate
    assert 2 * 24 * 6_000_000 < nbytes < 2 * 24 * 6_000_000 + 64 << 20
    bad = cpic.make_config(2, (128, 256), [1, 0, 0, 0], [0] * 4, [1, 1, 0, 0], 0.1, [(-1, 1, 1, 10)])
    with pytest.raises(cpic.CpicError) as e:
        cpic.Run.footprint(bad)
    assert "periodic" in str(e.value)
    odd = cpic.make_config(2, (33, 34), [1, 1, 0, 0], [0] * 4, [1, 1, 0, 0], 0.1, [(-1, 1, 1, 10)])
    with pytest.raises(cpic.CpicError):
        cpic.Run.footprint(odd)


def test_setters_reject_a_missing_run(lib_path):
    """The solver and push-tuning setters validate on the host: a NULL run is refused with
    CPIC_ERR_INVALID and a message, before any CUDA call."""
    from paper_1311_2286_gb300 import cpic

    lib = cpic.load(lib_path)
    assert lib.cpic_set_solver(None, cpic.CPIC_SOLVER_BICGSTAB) == cpic.CPIC_ERR_INVALID
    assert b"NULL" in lib.cpic_last_error()
    assert lib.cpic_set_push_tuning(None, 1024, 1) == cpic.CPIC_ERR_INVALID


def test_product_path_refuses_missing_library(tmp_path):
    from paper_1311_2286_gb300 import cpic

    saved = cpic._lib
    try:
        cpic._lib = None
        with pytest.raises(RuntimeError):
            cpic.load(str(tmp_path / "nope.so"))
    finally:
        cpic._lib = saved
