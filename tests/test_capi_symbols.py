"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/picasso.h declares (no compute calls here)."""
import ctypes

from paper_2401_06713_b300 import build as pbuild


def test_library_exports_header_symbols():
    path = pbuild.build()
    from paper_2401_06713_b300 import picasso

    names = picasso.header_symbols()
    assert "picasso_init" in names and "picasso_build_conflicts" in names and "picasso_color" in names
    lib = ctypes.CDLL(path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a binding signature (or is strerror)
    unbound = [n for n in names if n not in picasso._SIGS and n != "picasso_strerror"]
    assert not unbound, unbound


def test_strerror_and_defaults_without_gpu():
    from paper_2401_06713_b300 import picasso

    lib = picasso.lib()
    assert lib.picasso_strerror(0) == b"ok"
    assert b"budget" in lib.picasso_strerror(picasso.ERR_BUDGET)
    cfg = picasso.Config()
    assert lib.picasso_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.palette_num, cfg.palette_den, cfg.alpha) == (1, 8, 2.0)
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert lib.picasso_init(ctypes.byref(h), ctypes.byref(cfg), None, 10, 8, None) == picasso.ERR_INVALID_ARG
    assert lib.picasso_pack(None, 5, 1025, None, None) == picasso.ERR_UNSUPPORTED
    assert lib.picasso_pack(None, 5, 65, None, None) == picasso.ERR_INVALID_ARG
    assert lib.picasso_destroy(None) == picasso.ERR_INVALID_ARG
