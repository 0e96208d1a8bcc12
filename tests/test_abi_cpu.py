"""CPU checks of the C ABI: the library builds and exports every entry point
that include/gcamb.h declares, and its host-side logic (argument checks,
quadrature weights, active extents) is right without touching a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return gcamb.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "gcamb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gcamb_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert "gcamb_los_cl" in names and "gcamb_grid_create" in names
    raw = ctypes.CDLL(gcamb.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_version_and_error_text(L):
    assert "sm_103a" in gcamb.version()
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.grid_create([0.1, 0.05], [1.0, 2.0], 10.0, 2, 10)
    assert ei.value.code == gcamb.EINVAL
    assert "increasing" in gcamb.last_error()


@pytest.mark.parametrize("bad", [
    dict(k=[0.1, 0.2], tau=[1.0, 2.0], tau0=1.5, lmin=2, lmax=10),     # tau beyond tau0
    dict(k=[-0.1, 0.2], tau=[1.0, 2.0], tau0=3.0, lmin=2, lmax=10),    # k <= 0
    dict(k=[0.1, 0.2], tau=[2.0, 1.0], tau0=3.0, lmin=2, lmax=10),     # tau decreasing
    dict(k=[0.1, 0.2], tau=[1.0, 2.0], tau0=3.0, lmin=5, lmax=4),      # lmax < lmin
    dict(k=[0.1, 0.2], tau=[1.0, 2.0], tau0=3.0, lmin=2, lmax=30000),  # lmax too large
    dict(k=[], tau=[1.0, 2.0], tau0=3.0, lmin=2, lmax=10),             # empty k
])
def test_grid_create_rejects(L, bad):
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.grid_create(bad["k"], bad["tau"], bad["tau0"], bad["lmin"], bad["lmax"])
    assert ei.value.code == gcamb.EINVAL


def test_plain_c_client(L, tmp_path):
    """The header compiles as C99 with -pedantic and no warnings, and a plain
    C program linked against libgcamb.so (no Python, no torch) runs the
    host-side entry points as documented (tests/c_abi_host.c)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_host")
    libdir = os.path.dirname(gcamb.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_host.c"), "-L", libdir, "-lgcamb", "-lm",
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_table_compressed_argument_errors(L):
    """Host-side checks of gcamb_table_compressed: an unknown mode and a NULL
    pointer are EINVAL, a table that was never built is ESTATE."""
    wl = synth.workload("plain_lmax500")
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    out = ctypes.c_int(-1)
    assert L.gcamb_table_compressed(g.handle, 99, ctypes.byref(out)) == gcamb.EINVAL
    assert L.gcamb_table_compressed(g.handle, gcamb.F16X3, None) == gcamb.EINVAL
    assert L.gcamb_table_compressed(None, gcamb.F16X3, ctypes.byref(out)) == gcamb.EINVAL
    assert L.gcamb_table_compressed(g.handle, gcamb.F16X3, ctypes.byref(out)) == gcamb.ESTATE
    assert "build the table" in gcamb.last_error()
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.table_compressed(g, gcamb.PLAIN64)
    assert ei.value.code == gcamb.ESTATE
    gcamb.grid_destroy(g)


def test_weights_match_trapezoid(L, orc):
    wl = synth.workload("plain_lmax500")
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    wt, wk = gcamb.grid_weights(g)
    assert np.allclose(wt, orc.trapz_weights(wl.tau), rtol=1e-15, atol=0)
    assert np.allclose(wk, orc.lnk_weights(wl.k), rtol=1e-14, atol=0)
    info = gcamb.grid_info(g)
    assert info["nk"] == 300 and info["ntau"] == 400 and info["nl"] == 499 and info["n_ltile"] == 4


def test_extents_are_safe_and_tight(L, orc):
    """Beyond the stored prefix every multipole of the tile has |j_l| < eps_cut;
    at the last node inside it the tile's first multipole is not far below."""
    wl = synth.workload("plain_lmax500")
    eps = 1e-30
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, eps)
    ext = gcamb.grid_extents(g)
    nlt = ext.shape[1]
    # the prefix shrinks with the tile
    assert np.all(np.diff(ext, axis=1) <= 0)
    rng = np.random.default_rng(2)
    checked = 0
    for q in rng.integers(0, wl.nk, 40):
        for lt in range(nlt):
            l0 = wl.lmin + 128 * lt
            l1 = min(l0 + 127, wl.lmax)
            e = ext[q, lt]
            if e < wl.ntau:
                x = wl.k[q] * (wl.tau0 - wl.tau[e])
                j = orc.sph_bessel(l1, x)[l0:l1 + 1]
                assert np.abs(j).max() < eps
                checked += 1
            if e > 0:
                x = wl.k[q] * (wl.tau0 - wl.tau[e - 1])
                j = orc.sph_bessel(l0, x)[l0]
                assert abs(j) > eps * 1e-6
    assert checked > 20


def test_active_count_bounds_true_activity(L, orc):
    """The per-l Watson prefix counts every (l,k,tau) with |j_l| >= eps and
    not many more."""
    k = synth.log_grid(1e-4, 0.3, 40)
    tau = np.linspace(200.0, 14000.0, 120)
    lmax = 300
    g = gcamb.grid_create(k, tau, 14000.0, 2, lmax, 1e-30)
    info = gcamb.grid_info(g)
    x = (k[:, None] * (14000.0 - tau[None, :])).ravel()
    J = orc.sph_bessel(lmax, x)[:, 2:]
    true_active = int((np.abs(J) >= 1e-30).sum())
    assert info["active"] >= true_active
    assert info["active"] <= 1.25 * true_active
    assert info["stored_plain64"] >= info["active"]


def test_plan_info_fields_match_the_header():
    """The binding names as many plan-info fields as the header's
    GCAMB_PLAN_INFO_N, and reads that many (no short or long buffer)."""
    import inspect

    from paper_2509_25110_gb300 import gcamb
    txt = open(os.path.join(ROOT, "include", "gcamb.h")).read()
    n = int(re.search(r"#define\s+GCAMB_PLAN_INFO_N\s+(\d+)", txt).group(1))
    src = inspect.getsource(gcamb.plan_info)
    keys = re.search(r"keys\s*=\s*\(([^)]*)\)", src).group(1)
    assert len(re.findall(r'"(\w+)"', keys)) == n
    assert "(ctypes.c_int64 * %d)" % n in src
