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


def _lib():
    from paper_1802_04516_gb300 import binding, build
    return binding.load(build.build())


def _opts(**kw):
    from paper_1802_04516_gb300.binding import stdg_options
    o = stdg_options(p=2, p_gamma=2, scheme=1, precision=0, rel_tol=1e-8, max_iters=100, gmres_restart=20,
                     inner_tol=1e-4, use_graph=1, preconditioner=2)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_create_rejects_bad_options_before_touching_the_device():
    # every rejection happens on the host, before a stream or device buffer exists
    lib = _lib()
    bad = [dict(p=0), dict(p=5), dict(p_gamma=-1), dict(p_gamma=5), dict(scheme=2), dict(scheme=0, p_gamma=1),
           dict(precision=2), dict(preconditioner=3), dict(preconditioner=-1), dict(rel_tol=0.0),
           dict(rel_tol=float("nan")), dict(max_iters=0)]
    for kw in bad:
        out = ctypes.c_void_p(12345)
        assert lib.stdg_create(ctypes.byref(out), 2, ctypes.byref(_opts(**kw)), None) == -1, kw
        assert out.value is None, kw
    out = ctypes.c_void_p(12345)
    assert lib.stdg_create(ctypes.byref(out), 3, ctypes.byref(_opts(p=4, p_gamma=1)), None) == -1   # 3D: p <= 3
    for dim in (1, 4):
        assert lib.stdg_create(ctypes.byref(out), dim, ctypes.byref(_opts()), None) == -1
    assert lib.stdg_create(None, 2, ctypes.byref(_opts()), None) == -1
    assert lib.stdg_create(ctypes.byref(out), 2, None, None) == -1


def test_every_call_rejects_a_null_context():
    from paper_1802_04516_gb300.binding import SIGNATURES
    lib = _lib()
    lib.stdg_destroy(None)                                   # a no-op
    assert lib.stdg_last_error(None) == b"null context"
    assert lib.stdg_mesh_faces(2, 0, None, 0, None, None, None, None, None) == -1
    assert lib.stdg_measure_fma_peak(1, None) == -1           # null output, before touching the device
    for name, (res, args) in SIGNATURES.items():
        if name in ("stdg_create", "stdg_destroy", "stdg_last_error", "stdg_mesh_faces", "stdg_locate_points",
                    "stdg_reference_tables", "stdg_measure_fma_peak"):
            continue                                         # no context argument
        vals = [None] + [a(0) if a in (ctypes.c_int, ctypes.c_int64, ctypes.c_double) else None for a in args[1:]]
        assert getattr(lib, name)(*vals) == -1, name
