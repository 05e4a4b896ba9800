"""The Python binding checks every array it hands to the library against the context's
sizes before the call (the C functions read or write exactly that many values through
the pointer).  CPU: a stand-in library records calls; no GPU, no context."""
import numpy as np
import pytest

from paper_1802_04516_gb300 import binding


class _Lib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            return 0
        return f


class _Solver(binding.Solver):
    SIZES = {0: 10, 1: 16, 2: 6, 3: 6, 4: 3, 5: 3, 6: 2, 7: 10 * 2 * 3 * 6}

    def __init__(self):                       # no library context
        self.lib, self.h, self.dim, self.n_rec = _Lib(), 1, 2, 4

    def query(self, what):
        return self.SIZES[what]


def test_sizes_are_checked_before_the_call():
    s = _Solver()
    ne, nf = 10, 16
    good_v, good_s = np.zeros((ne, 2, 6)), np.zeros((nf, 3, 6))
    s.set_state(good_v, good_s)
    s.set_material(np.ones(ne), np.ones(ne), np.ones(ne))
    s.apply_operator(0.1, np.zeros(360))
    s.set_sources(np.zeros((2, 2)), np.zeros((2, 2)), 1.0, 0.1, 1.0)
    s.set_point_sources(np.zeros((4, 2)), np.zeros((4, 2)), 1.0, 0.1, 1.0, n_shots=2)
    s.misfit_grad(0.1, 5, np.zeros((2, 5, 4, 2)))
    s.get_state(out=(np.zeros((ne, 2, 6)), np.zeros((nf, 3, 6))))
    n_ok = len(s.lib.calls)
    bad = [
        lambda: s.set_state(np.zeros((ne, 2, 5)), good_s),
        lambda: s.set_state(good_v, np.zeros((nf - 1, 3, 6))),
        lambda: s.set_material(np.ones(ne - 1), np.ones(ne), np.ones(ne)),
        lambda: s.apply_operator(0.1, np.zeros(359)),
        lambda: s.apply_preconditioner(0.1, np.zeros(361)),
        lambda: s.set_sources(np.zeros((2, 3)), np.zeros((2, 3)), 1.0, 0.1, 1.0),
        lambda: s.set_point_sources(np.zeros((3, 2)), np.zeros((3, 2)), 1.0, 0.1, 1.0, n_shots=2),
        lambda: s.set_receivers(np.zeros((4, 3))),
        lambda: s.set_plane_wave(0, [1.0, 0.0, 0.0]),
        lambda: s.misfit_grad(0.1, 5, np.zeros((2, 4, 4, 2))),
        lambda: s.get_state(out=(np.zeros((ne, 2, 6), dtype=np.float32), np.zeros((nf, 3, 6)))),
        lambda: s.get_state(out=(np.zeros((ne, 2, 6)), np.zeros((nf, 3, 5)))),
    ]
    for k, f in enumerate(bad):
        with pytest.raises(ValueError):
            f()
        assert len(s.lib.calls) == n_ok, k                  # nothing reached the library
