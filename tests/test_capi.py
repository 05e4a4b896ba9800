"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU)."""
import ctypes

from helpers import header_functions


def test_library_builds_and_exports_header_symbols():
    from paper_1802_04516_gb300 import binding, build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.exported_symbols()) == declared


def test_options_struct_layout():
    from paper_1802_04516_gb300.binding import stdg_options, stdg_stats
    # int p, p_gamma, scheme, precision; double rel_tol; int max_iters, gmres_restart; double inner_tol;
    # int use_graph, preconditioner
    assert ctypes.sizeof(stdg_options) == 48
    assert ctypes.sizeof(stdg_stats) == 32
