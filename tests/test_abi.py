"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
function include/pivbos.h declares, agrees with the binding on struct
layouts, and rejects bad arguments before touching the device."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pivbos.h")
TESTING_HEADER = os.path.join(ROOT, "include", "pivbos_testing.h")


@pytest.fixture(scope="module")
def P():
    from paper_1812_05902_gb300 import build
    build.build()
    from paper_1812_05902_gb300 import pivbos
    return pivbos


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pivbos_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(P):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(P.lib(), n), n
        assert n in P.EXPORTED, n
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(pivbos_\w+)", out))
    assert set(names) <= exported


def test_testing_hooks_live_in_their_own_library(P):
    """The checking and measurement hooks are declared in pivbos_testing.h and
    exported by libpivbos_testing.so, not by the product library."""
    names = declared_functions(TESTING_HEADER)
    assert set(names) == set(P.TESTING_EXPORTED)
    T = P.testing_lib()
    for n in names:
        assert hasattr(T, n), n
    product = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    testing = subprocess.run(["nm", "-D", "--defined-only", P.TESTING_LIB_PATH], capture_output=True,
                             text=True).stdout
    assert set(names) <= set(re.findall(r"\sT\s(pivbos_\w+)", testing))
    assert not set(names) & set(re.findall(r"\sT\s(pivbos_\w+)", product))
    assert not set(names) & set(declared_functions(HEADER))


def test_struct_layouts_match_header(P):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "pivbos.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pivbos_surface),
         offsetof(pivbos_surface, clear_radius), sizeof(pivbos_ray_state), offsetof(pivbos_ray_state, status),
         sizeof(pivbos_frame_desc), offsetof(pivbos_frame_desc, stats), sizeof(pivbos_tuning),
         sizeof(pivbos_surrogate_cfg), offsetof(pivbos_surrogate_cfg, ref_plane_z),
         sizeof(pivbos_surrogate_report), offsetof(pivbos_surrogate_report, target_rms));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals[0] == ctypes.sizeof(P.pivbos_surface)
    assert vals[1] == P.pivbos_surface.clear_radius.offset
    assert vals[2] == P.RAY_STATE.itemsize
    assert vals[3] == P.RAY_STATE.fields["status"][1]
    assert vals[4] == ctypes.sizeof(P.pivbos_frame_desc)
    assert vals[5] == P.pivbos_frame_desc.stats.offset
    assert vals[6] == ctypes.sizeof(P.pivbos_tuning)
    assert vals[7] == ctypes.sizeof(P.pivbos_surrogate_cfg)
    assert vals[8] == P.pivbos_surrogate_cfg.ref_plane_z.offset
    assert vals[9] == ctypes.sizeof(P.pivbos_surrogate_report)
    assert vals[10] == P.pivbos_surrogate_report.target_rms.offset


def test_surrogate_arguments_without_a_device(P):
    L = P.lib()
    assert L.pivbos_surrogate_default_cfg(None) == P.ERR_INVALID_ARG
    cfg = P.pivbos_surrogate_default_cfg()
    assert cfg.n_train == 20_000_000 and cfg.batch == 16384 and np.isnan(cfg.ref_plane_z)
    assert cfg.born_segments == -1 and cfg.use_network == -1
    assert abs(cfg.err_budget_px - 0.01) < 1e-9
    out = ctypes.c_void_p()
    rep = P.pivbos_surrogate_report()
    assert L.pivbos_surrogate_train(None, 1, None, ctypes.byref(out), None, None) == P.ERR_INVALID_ARG
    fake = ctypes.c_void_p(1)  # never dereferenced: the configuration check fails first
    desc = P.pivbos_frame_desc(fake, fake, fake, 1, 1, 0, 0, 1e-4, fake, None)
    no_medium = P.pivbos_frame_desc(None, fake, fake, 1, 1, 0, 0, 1e-4, fake, None)
    assert L.pivbos_surrogate_train(ctypes.byref(no_medium), 1, None, ctypes.byref(out), None,
                                    None) == P.ERR_INVALID_ARG
    for field, value in (("batch", 100), ("batch", 1 << 17), ("n_train", 10), ("epochs", 0), ("lr", 0.0),
                         ("err_budget_px", -1.0), ("budget_margin", 1.5), ("min_bin_count", 0),
                         ("ref_plane_z", float("inf")), ("born_segments", -2), ("born_segments", 65),
                         ("use_network", 2), ("use_network", -2), ("table_columns_per_cell", -1), ("table_columns_per_cell", 9),
                         ("table_levels_per_cell", 5)):
        bad = P.pivbos_surrogate_default_cfg()
        setattr(bad, field, value)
        assert L.pivbos_surrogate_train(ctypes.byref(desc), 1, ctypes.byref(bad), ctypes.byref(out),
                                        ctypes.byref(rep), None) == P.ERR_INVALID_ARG, field
        assert "configuration" in P.pivbos_last_error()
    assert L.pivbos_surrogate_render(None, ctypes.byref(desc), None, None) == P.ERR_INVALID_ARG
    assert L.pivbos_surrogate_sensor(None, ctypes.byref(desc), None, 0, None, None, None, None) == P.ERR_INVALID_ARG
    assert L.pivbos_surrogate_report_get(None, ctypes.byref(rep)) == P.ERR_INVALID_ARG
    L.pivbos_surrogate_destroy(None)


def test_argument_errors_without_a_device(P):
    L = P.lib()
    out = ctypes.c_void_p()
    # optics
    assert L.pivbos_optics_create(None, -1, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 0, 2.0, 1e-5, 64, 64,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_create(None, 0, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 2, 2.0, 1e-5, 64, 64,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_create(None, 0, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 0, 2.0, 1e-5, 0, 64,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_create(None, 0, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 0, 2.0, 1e-5, 64, 64,
                                  None) == P.ERR_INVALID_ARG
    bad = (P.pivbos_surface * 1)(P.pivbos_surface(7, 0, 1.0, 0.1, 0.0, 1.5, 0.01))
    assert L.pivbos_optics_create(bad, 1, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 0, 2.0, 1e-5, 64, 64,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert "surface 0" in P.pivbos_last_error()
    # medium
    rho = np.ones(8, dtype=np.float32)
    o3 = (ctypes.c_double * 3)(0, 0, 0)
    h3 = (ctypes.c_double * 3)(1e-3, 1e-3, 1e-3)
    assert L.pivbos_medium_create(rho.ctypes.data, 0, 1, 2, 2, o3, h3, 0.2e-3, None,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_medium_create(None, 0, 2, 2, 2, o3, h3, 0.2e-3, None, ctypes.byref(out)) == P.ERR_INVALID_ARG
    hbad = (ctypes.c_double * 3)(1e-3, 0.0, 1e-3)
    assert L.pivbos_medium_create(rho.ctypes.data, 0, 2, 2, 2, o3, hbad, 0.2e-3, None,
                                  ctypes.byref(out)) == P.ERR_INVALID_ARG
    # render
    img = np.zeros(4, dtype=np.int64)
    src = np.zeros(3)
    assert L.pivbos_render(None, None, src.ctypes.data, 1, 0, 1, 0, 0, 0, 1e-4, img.ctypes.data, 0, None,
                           None) == P.ERR_INVALID_ARG
    fake = ctypes.c_void_p(1)  # never dereferenced: the count checks fail first
    assert L.pivbos_render(None, fake, src.ctypes.data, -1, 0, 1, 0, 0, 0, 1e-4, img.ctypes.data, 0, None,
                           None) == P.ERR_INVALID_ARG
    assert L.pivbos_render(None, fake, src.ctypes.data, 1, 0, 1, 0, 0, 5, 1e-4, img.ctypes.data, 0, None,
                           None) == P.ERR_INVALID_ARG
    assert L.pivbos_render(None, fake, src.ctypes.data, 1, 0, 1, 0, 0, 0, 0.0, img.ctypes.data, 0, None,
                           None) == P.ERR_INVALID_ARG
    assert L.pivbos_render(None, fake, src.ctypes.data, 1 << 20, 0, 1 << 12, 0, 0, 0, 1e-4,
                           img.ctypes.data, 0, None, None) == P.ERR_OVERFLOW
    assert L.pivbos_render(None, fake, src.ctypes.data, 1, 0, 1, 0, 0, 0, 1e-4, None, 0, None,
                           None) == P.ERR_INVALID_ARG
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    assert L.pivbos_timing_read(None, ctypes.byref(ms), ctypes.byref(n)) == P.ERR_INVALID_ARG
    assert L.pivbos_image_finalize(None, -1, None, None) == P.ERR_INVALID_ARG
    assert L.pivbos_image_finalize(None, 0, None, None) == P.OK
    # spot too wide for the window
    assert L.pivbos_optics_create(None, 0, 1.0, 1.0, 0.01, 64.0, 1.0, 5e-7, 0, 2.0, 1e-6, 64, 64,
                                  ctypes.byref(out)) == P.ERR_UNSUPPORTED


def test_bos_arguments_without_a_device(P):
    L = P.lib()
    fake = ctypes.c_void_p(1)  # never dereferenced: the argument checks fail first
    assert L.pivbos_bos_displacements(None, fake, fake, 1, 1, 0, 0, 1, 1e-4, None, None, None,
                                      None) == P.ERR_INVALID_ARG
    assert L.pivbos_bos_displacements(fake, fake, fake, 1, (1 << 22) + 1, 0, 0, 1, 1e-4, None, None, None,
                                      None) == P.ERR_UNSUPPORTED
    assert L.pivbos_bos_displacements(fake, None, fake, 1, 1, 0, 0, 1, 1e-4, None, None, None,
                                      None) == P.ERR_INVALID_ARG
    assert L.pivbos_bos_displacements(fake, fake, fake, 1, 1, 0, 0, 7, 1e-4, None, None, None,
                                      None) == P.ERR_INVALID_ARG
    assert L.pivbos_bos_theory(None, fake, fake, 1, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_bos_theory(fake, None, fake, 1, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_bos_theory(fake, fake, fake, -1, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, -1, 4, 4, 0.0, 0.0, 1.0, 0.0, fake, None,
                                    None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, (1 << 23) + 1, 4, 4, 0.0, 0.0, 1.0, 0.0, fake, None,
                                    None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, 1, 1, 4, 0.0, 0.0, 1.0, 0.0, fake, None,
                                    None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, 1, 4, 4, 0.0, 0.0, 0.0, 0.0, fake, None,
                                    None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, 1, 4, 4, 0.0, float("nan"), 1.0, 0.0, fake, None,
                                    None) == P.ERR_INVALID_ARG
    assert L.pivbos_regrid_bilinear(fake, fake, 1, 4, 4, 0.0, 0.0, 1.0, -1.0, fake, None,
                                    None) == P.ERR_INVALID_ARG


def test_optics_extension_arguments_without_a_device(P):
    L = P.lib()
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(1)
    assert L.pivbos_optics_tilt_sensor(None, 0.1, 0.0, ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_tilt_sensor(fake, float("inf"), 0.0, ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_tilt_sensor(fake, 0.1, 0.0, None) == P.ERR_INVALID_ARG
    # a lens array needs a positive pitch and a focal length; type 6 does not exist
    for row in ((P.SURF_LENS_ARRAY, 0, 1.0, 0.0, 0.01, 1.0, 0.05), (P.SURF_LENS_ARRAY, 0, 1.0, 1e-3, 0.0, 1.0, 0.05),
                (6, 0, 1.0, 0.0, 0.0, 1.0, 0.05)):
        bad = (P.pivbos_surface * 1)(P.pivbos_surface(*row))
        assert L.pivbos_optics_create(bad, 1, 1.0, 1.0, 0.01, 8.0, 0.1, 5e-7, 0, 2.0, 1e-5, 64, 64,
                                      ctypes.byref(out)) == P.ERR_INVALID_ARG


def test_pairs_arguments_without_a_device(P):
    L = P.lib()
    fake = ctypes.c_void_p(1)
    o3 = (ctypes.c_double * 3)(0, 0, 0)
    h3 = (ctypes.c_double * 3)(1e-3, 1e-3, 1e-3)
    bad = (ctypes.c_double * 3)(1e-3, 0.0, 1e-3)
    assert L.pivbos_advect_sources(fake, -1, fake, 4, 4, 4, o3, h3, 1e-3, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_advect_sources(fake, 1, fake, 1, 4, 4, o3, h3, 1e-3, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_advect_sources(fake, 1, fake, 4, 4, 4, o3, bad, 1e-3, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_advect_sources(fake, 1, fake, 4, 4, 4, o3, h3, float("nan"), fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_advect_sources(fake, 0, fake, 4, 4, 4, o3, h3, 1e-3, fake, None) == P.OK
    assert L.pivbos_image_u16(fake, -1, 1.0, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_image_u16(fake, 4, 0.0, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_image_u16(fake, 4, 1.0, fake, None) == P.ERR_INVALID_ARG     # misaligned
    assert L.pivbos_image_u16(fake, 0, 1.0, fake, None) == P.OK
    assert L.pivbos_mie(-1.0, 5e-7, 1.0, 1.5, 0.0, 10, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_mie(1e-6, 5e-7, 1.0, 1.5, 0.0, 1, fake, None) == P.ERR_INVALID_ARG
    assert L.pivbos_mie(1e-6, 5e-7, 1.0, 1.5, -0.1, 10, fake, None) == P.ERR_INVALID_ARG
    out = ctypes.c_void_p()
    L3 = (ctypes.c_double * 3)(1, 0, 0)
    assert L.pivbos_optics_radiance(None, L3, None, fake, 10, ctypes.byref(out)) == P.ERR_INVALID_ARG
    assert L.pivbos_optics_radiance(fake, L3, None, fake, 1, ctypes.byref(out)) == P.ERR_INVALID_ARG


def test_selftest_arguments_without_a_device(P):
    L = P.lib()
    assert L.pivbos_selftest_wait_timeout(0, None) == P.ERR_INVALID_ARG
    assert L.pivbos_selftest_wait_timeout((1 << 20) + 1, None) == P.ERR_INVALID_ARG


def _declared_arity(header=HEADER):
    """Parameter count of every function the header declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(pivbos_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_the_header(P):
    """The ctypes argument lists of the binding have as many parameters as
    the header's declarations (an ABI drift would misplace arguments)."""
    arity = _declared_arity()
    assert len(arity) >= 38
    L = P.lib()
    for name, n in arity.items():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
    T = P.testing_lib()
    for name, n in _declared_arity(TESTING_HEADER).items():
        f = getattr(T, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
