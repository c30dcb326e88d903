"""The C-ABI library loads on a CPU-only host and exports every entry point
declared in include/bdg.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bdg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_calls_of_the_boundary():
    names = declared_functions()
    for want in ("bdg_create", "bdg_destroy", "bdg_last_error", "bdg_build", "bdg_heev_workspace", "bdg_heev",
                 "bdg_refine", "bdg_densities", "bdg_scf_step", "bdg_heev_batched"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2310_03341_b300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_lists_the_same_symbols():
    import paper_2310_03341_b300 as bdg
    assert sorted(bdg.EXPORTS) == declared_functions()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2310_03341_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "bdg_oracle" not in txt, f


def test_fno_parameter_count_matches_the_reference_layout():
    """bdg_fno_sizes is host-only: its parameter count equals the layout of oracle/fno.py."""
    import ctypes as C
    import paper_2310_03341_b300 as bdg
    from oracle import fno as ofno
    for (g, w, m, L) in [(8, 32, 4, 4), (6, 8, 2, 3), (24, 32, 8, 4)]:
        cfg = bdg.FnoConfig(g, w, m, L, 5, 3, 1)
        npar, ncache = C.c_int64(), C.c_int64()
        assert bdg.lib().bdg_fno_sizes(C.byref(cfg), 2, C.byref(npar), C.byref(ncache)) == 0
        assert npar.value == ofno.sizes(g, w, m, L, 5, 3)[0]
        M = (2 * m - 1) ** 3
        assert ncache.value == L * (2 * 2 * g ** 3 * w + 2 * M * w * 2) + 2 * g ** 3 * w


def test_argument_checks_that_need_no_device():
    """Null contexts and the fixed scratch limit are refused before any CUDA call."""
    import ctypes as C
    import paper_2310_03341_b300 as bdg
    L = bdg.lib()
    assert L.bdg_last_error(None) == b"null context"
    assert L.bdg_heev(None, 4, None, 4, None, None, 4, 0, None) == bdg.ERRORS_BY_NAME["EINVAL"]
    assert L.bdg_heev_batched(None, 0, None, None, None, None, 0, None) == bdg.ERRORS_BY_NAME["EINVAL"]
    assert L.bdg_refine(None, None, 0.0, None, None, 4, None, None, 4, 1, 1e-10, None, None, None, None) == \
        bdg.ERRORS_BY_NAME["EINVAL"]
    g = bdg.Grid(56, 56, 56, 1.0)                    # V = 175616 sites > 174720
    msg = C.create_string_buffer(256)
    rc = L.bdg_densities_noalloc(C.byref(g), 2 * 56 ** 3, C.c_void_p(16), C.c_void_p(16), 2 * 56 ** 3, 0.0, 1.0,
                                 C.c_void_p(16), C.c_void_p(16), None, msg, 256)
    assert rc == bdg.ERRORS_BY_NAME["EUNSUPPORTED"]
    assert b"scratch limit" in msg.value
