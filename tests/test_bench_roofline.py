"""bench.py's roofline arithmetic on CPU (a stand-in solver returns fixed launch times):
algorithmic bytes per launch of the FP32 face kernel and the Pre2 local step for the
200,704-triangle p = p_gamma = 3 benchmark mesh, counted by hand from the data each
launch must move; achieved = bytes / time, frac = achieved / peak; the ncu per-unit
traffic scaled to the launch; the dominant kernel chosen by device time per Krylov
iteration; DOFs per slab."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N_ELEM, N_FACE = 200704, 301728


class _Timed:
    def __init__(self, ms_op, ms_kernel, pre2_bits=32):
        self.ms_op, self.ms_kernel, self.pre2_bits = ms_op, ms_kernel, pre2_bits

    def time_operator(self, dt, fp32, n):
        return self.ms_op

    def time_kernel(self, dt, which, fp32, n):
        assert which == 2 and fp32
        return self.ms_kernel


def _w(p=3, pg=3):
    return types.SimpleNamespace(dim=2, p=p, p_gamma=pg, n_elem=N_ELEM, dt=1e-3)


def test_face_kernel_bytes_and_fraction():
    # per face: two 2 x 10 x 10 FP32 blocks of D~ (1600 B), lambda and mu (8 B), two
    # element ids (8 B); per launch: x read, y read and written (3 x 4 B x 16,056,320)
    nvel = N_ELEM * 2 * 4 * 10
    assert nvel == 16056320
    alg = N_FACE * (1600 + 8 + 8) + 3 * 4 * nvel
    r = bench.face_kernel_roofline(_Timed(0.5, None), _w(), True, N_FACE, {"hbm_gbs": 8000.0})
    assert r["alg_bytes_per_launch"] == alg == 680268288
    assert abs(r["achieved"] - alg / 0.5e-3 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 8000.0) < 1e-4 and r["peak_source"] == "measured hbm_gbs"
    # ncu's DRAM bytes per face of the tiled kernel on the 102,400-triangle copy, scaled
    assert r["traffic"] == int((344876032 + 27466752) / 154080 * N_FACE)
    assert bench.face_kernel_roofline(_Timed(0.5, None), _w(), True, N_FACE, {})["peak_source"] == "fallback"


def test_pre2_local_bytes_and_fraction():
    # per element one dense 80 x 80 FP32 block (N = d N_phi N_gamma = 80) plus r, w read, z written
    N = 2 * 10 * 4
    alg = N_ELEM * N * N * 4 + 3 * 4 * N_ELEM * N
    r = bench.pre2_local_roofline(_Timed(None, 0.8), _w(), {"hbm_gbs": 7000.0})
    assert r["alg_bytes_per_launch"] == alg == 5330698240
    assert abs(r["achieved"] - alg / 0.8e-3 / 1e9) < 0.1 and abs(r["frac"] - r["achieved"] / 7000.0) < 1e-4
    assert r["traffic"] == int((429949184 + 2444032) / 16384 * N_ELEM)
    # the ncu per-unit figures belong to the p = 3 shape only
    assert bench.pre2_local_roofline(_Timed(None, 0.8), _w(2, 2), {"hbm_gbs": 7000.0})["traffic"] is None


def test_pre2_local_bytes_with_fp16_blocks():
    # balanced FP16 storage: N^2 FP16 entries and 2N FP32 scales per element, same vectors
    N = 80
    alg = N_ELEM * (N * N * 2 + 2 * N * 4) + 3 * 4 * N_ELEM * N
    r = bench.pre2_local_roofline(_Timed(None, 0.45, pre2_bits=16), _w(), {"hbm_gbs": 7000.0})
    assert r["alg_bytes_per_launch"] == alg and r["kernel"] == "pre2_local_half_kernel"
    assert abs(r["achieved"] - alg / 0.45e-3 / 1e9) < 0.1
    # ncu's DRAM bytes per element of the FP16 kernel on the 102,400-triangle copy, scaled
    assert r["traffic"] == int((1450097000 + 32895744) / 102400 * N_ELEM)


def test_dominant_kernel_by_time_per_iteration():
    cands = {"face": {"ms_per_launch": 0.38}, "pre2_local": {"ms_per_launch": 0.70}}
    assert bench.dominant_roofline(cands, {"face": 1, "pre2_local": 1})["ms_per_launch"] == 0.70
    d = bench.dominant_roofline(cands, {"face": 2, "pre2_local": 1})
    assert d["ms_per_launch"] == 0.38 and d["launches_per_krylov_iteration"] == 2


def test_dofs_per_slab():
    w = types.SimpleNamespace(dim=2, p=3, p_gamma=3, n_elem=N_ELEM)
    # velocity d N_phi N_gamma per element + stress s N_psi N_gamma per face (N_psi = N_phi)
    assert bench.dofs_per_slab(w, N_FACE) == N_ELEM * 2 * 10 * 4 + N_FACE * 3 * 10 * 4 == 52263680


def test_velocity_dofs_per_slab():
    w = types.SimpleNamespace(dim=2, p=3, p_gamma=3, n_elem=N_ELEM)
    assert bench.velocity_dofs_per_slab(w) == N_ELEM * 2 * 10 * 4 == 16056320
    w3 = types.SimpleNamespace(dim=3, p=2, p_gamma=2, n_elem=1000)
    assert bench.velocity_dofs_per_slab(w3) == 1000 * 3 * 10 * 3
