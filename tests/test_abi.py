"""The C-ABI library builds, loads and exports every entry point declared in include/*.h (CPU only)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dh_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2512_13403_b300 import _lib, build
    build.build()
    lib = _lib.load()
    declared = _declared()
    assert {"dh_create", "dh_step", "dh_advance", "dh_init_state", "dh_adjoint_advance"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly the header's functions
    assert set(_lib.exported_names()) == declared


def test_config_struct_matches_header_layout():
    import ctypes as C
    from paper_2512_13403_b300 import _lib
    lib = _lib.load()
    cfg = _lib.DhConfig()
    lib.dh_config_default(C.byref(cfg), 16, 8, 4)
    assert (cfg.nx, cfg.ny, cfg.nz) == (16, 8, 4)
    assert cfg.dx == 1 / 16 and cfg.dz == 1 / 4
    assert abs(cfg.gamma - 5 / 3) < 1e-15 and cfg.cfl == 0.4
    assert cfg.ou_tau == 0.5 and cfg.t_floor == 0.05 and cfg.mg_tol == 1e-6
    assert cfg.mg_pre == 2 and cfg.mg_post == 2 and cfg.nsub_max == 1024
    # the fields after the mg sweep counts (offsets follow the header's order)
    assert cfg.mg_smoother == 0 and abs(cfg.mg_omega - 2 / 3) < 1e-15 and cfg.mg_cycle == 1
    assert cfg.limiter == 0 and cfg.integrator == 2
    assert cfg.c_cool == float("inf")   # the last field: the cooling time-step limit is off


def test_create_rejects_bad_config_without_gpu_work():
    """Validation happens before any device call, so it is checkable on the CPU."""
    import ctypes as C
    from paper_2512_13403_b300 import _lib
    lib = _lib.load()
    cfg = _lib.DhConfig()
    lib.dh_config_default(C.byref(cfg), 2, 8, 8)
    ctx = C.c_void_p()
    assert lib.dh_create(C.byref(cfg), None, C.byref(ctx)) == _lib.DH_ERR_ARG
    assert b">= 4" in lib.dh_last_error(None)
    assert lib.dh_status_string(_lib.DH_ERR_POSITIVITY) == b"DH_ERR_POSITIVITY"
    for field, bad, msg in (("mg_cycle", 3, b"mg_cycle"), ("mg_smoother", 2, b"mg_smoother"),
                            ("mg_omega", 1.5, b"mg_omega"), ("limiter", 2, b"limiter"),
                            ("integrator", 4, b"integrator"), ("c_cool", 0.0, b"c_cool"),
                            ("c_cool", -1.0, b"c_cool")):
        lib.dh_config_default(C.byref(cfg), 16, 16, 16)
        cfg.gravity = 1
        setattr(cfg, field, bad)
        assert lib.dh_create(C.byref(cfg), None, C.byref(ctx)) == _lib.DH_ERR_ARG
        assert msg in lib.dh_last_error(None)
