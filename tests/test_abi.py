"""The C ABI library builds, loads and exports every entry point include/wf.h declares.
Host-only calls; no GPU needed."""
import ctypes
import os
import re

import pytest

import paper_0906_3978_gb300 as wf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    wf.build()
    return wf.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z_]+)\s*\(", src)))


def test_header_declares_boundary():
    names = declared_functions()
    for required in ["wf_create", "wf_destroy", "wf_grid_assign", "wf_build_noise", "wf_solve",
                     "wf_solve_batch", "wf_submit", "wf_poll", "wf_status_string", "wf_set_fused_planes",
                     "wf_smooth", "wf_compare", "wf_density_stats", "wf_selection_eval",
                     "wf_grid_assign_weighted", "wf_rsd_factor", "wf_deconvolve", "wf_sd_noise",
                     "wf_jackknife_masses", "wf_project_mask", "wf_solve_response", "wf_jackknife_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for s in [0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9]:
        assert wf.status_string(s) and wf.status_string(s) != "unknown status"
    assert wf.status_string(42) == "unknown status"


def test_supported_sizes(lib):
    for n in [16, 24, 32, 48, 64, 72, 96, 108, 128, 144, 192, 216, 256, 288, 384, 512]:
        assert wf.supported_size(n)
    for n in [0, 8, 20, 100, 1000, 1024, -4]:
        assert not wf.supported_size(n)


def test_rsd_factor_matches_oracle():
    """The library's closed form (host code) against the oracle's quadrature of the definition,
    across the switch between the power series and the arctan form (k^2 sigma_v^2 / 2 = 1/2)."""
    import numpy as np
    import paper_0906_3978_gb300 as wf
    from oracle import evaluation as ev
    k = np.concatenate([[0.0, 1e-4], np.linspace(0.01, 0.5, 30), [0.1999, 0.2, 0.2001], np.linspace(0.6, 6.0, 20)])
    for beta in (0.0, 0.42, 1.3):
        got, ref = wf.rsd_factor(k, beta, 5.0), ev.rsd_factor(k, beta, 5.0)
        assert np.max(np.abs(got - ref) / ref) <= 5e-14
    for bad in (dict(k=[-1.0]), dict(k=[np.nan]), dict(sigma_v=-1.0)):
        a = dict(k=[0.1], beta=0.4, sigma_v=5.0)
        a.update(bad)
        with pytest.raises(wf.WfError):
            wf.rsd_factor(a["k"], a["beta"], a["sigma_v"])


def test_product_path_never_loads_the_oracle():
    """The library and its binding stand alone: importing and building them loads no part of the
    oracle, and no source of the package or the header refers to it."""
    import subprocess
    import sys
    code = ("import sys; import paper_0906_3978_gb300 as wf; wf.build(); wf.lib(); "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True, timeout=600)
    pkg = os.path.join(ROOT, "paper_0906_3978_gb300")
    for d, _, files in os.walk(pkg):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(d, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|liboracle|oracle\.c", src, re.M), f


def test_header_is_plain_c_and_links(lib):
    """include/wf.h compiles as strict C11 without warnings, and a C program links against the
    library and calls a host-only entry point (no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    d = os.path.join(ROOT, "paper_0906_3978_gb300", "_build", "ctest")
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "use.c")
    with open(src, "w") as f:
        f.write('#include "wf.h"\n#include <stdio.h>\n'
                'int main(void) { printf("%s %d\\n", wf_status_string(WF_ERR_ARG), wf_supported_size(384)); '
                'return 0; }\n')
    libdir = os.path.join(ROOT, "paper_0906_3978_gb300")
    exe = os.path.join(d, "use")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        src, "-L", libdir, "-lwf", "-Wl,-rpath," + libdir, "-o", exe],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.split() == ["invalid", "argument", "1"]


def test_automatic_coarse_radius(lib):
    """deflate = -1's radius by grid size for mixed solves (none for FP64), within its limits
    (1 <= K <= 12, 4 K < n) wherever it is not 0."""
    want = {16: 0, 32: 0, 48: 0, 64: 3, 96: 4, 128: 4, 192: 6, 256: 8, 384: 10, 512: 12}
    for n, k in want.items():
        assert wf.deflate_radius(n) == k, n
        assert wf.deflate_radius(n, wf.FP64) == 0
    for n in range(16, 513, 8):
        k = wf.deflate_radius(n)
        assert k == 0 or (1 <= k <= 12 and 4 * k < n), n
