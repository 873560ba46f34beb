"""CPU-side checks of the C ABI library (no kernel is launched here)."""
import ctypes
import re

import paper_1403_4781_gb300 as sdl


def test_library_loads_and_exports_every_declared_symbol():
    lib = sdl.lib()
    names = sdl.declared_symbols()
    assert {"sdl_omp", "sdl_mod_update", "sdl_local_train", "sdl_merge"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1403_4781_gb300 import _SIGS
    assert set(_SIGS) == set(sdl.declared_symbols())


def test_null_context_and_bad_arguments_are_rejected_without_a_gpu():
    lib = sdl.lib()
    # NULL context -> SDL_EINVAL, nothing launched
    assert lib.sdl_omp(None, 1, None, 64, 256, None, 10, 6, 0.0, None, None, None, None) == 1
    assert lib.sdl_destroy(None) == 0
    h = ctypes.c_void_p()
    assert lib.sdl_corr_features(None, None, 64, 256, None, None, 1, None) == 1
    assert lib.sdl_omp_proposed_batched(None, None, 1, None, 64, 256, None, None, 1, 6, 12, 0.1,
                                        None, None, None, None, None) == 1
    # no CUDA device in this container: sdl_create must fail cleanly, not crash
    rc = lib.sdl_create(ctypes.byref(h), 0, None)
    assert rc in (0, 1, 4)
    if rc == 0:
        lib.sdl_destroy(h)


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    import os
    with open(os.path.join(sdl._build.INCLUDE, "sdl.h")) as f:
        text = f.read()
    for name in ("sdl_omp", "sdl_mod_update", "sdl_split", "sdl_local_train", "sdl_merge",
                 "sdl_residual", "sdl_recovery", "sdl_init_dict"):
        pos = text.index(name + "(")
        block = text[max(0, text.rfind("/*", 0, pos)):pos]
        assert re.search(r"Sec\.|Algorithm|Table|Def\.", block), name
