"""The paper's printed tables (fixtures under tests/golden/, each citing its table)
against the readings that the oracle and the tests take from them (CPU, no solves).

* Table 1 (Sec. 6.2) prints five mesh sizes h for four meshes, 0.0842 twice.  Reading:
  h_k = 0.1264 sqrt(1760 / N_k) = (0.1264, 0.0842, 0.0632, 0.0505).  Under it every
  printed rate equals log(e_k / e_(k+1)) / log(h_k / h_(k+1)) to its printed digit; the
  printed list taken in order cannot give them (a zero step from 0.0842 to 0.0842).
* Table 1: on the finest pair of meshes every variable converges at p + 1 or better,
  the order the convergence tests of the oracle (CPU) and of the GPU path require.
* The sliver table (Sec. 6.5): the factor column is mesh 2 over mesh 1, Pre2 keeps the
  iteration count mesh-independent and the ordering none > Pre1 > Pre2 holds on both
  meshes; the GPU sliver study checks the same ordering on its own meshes.
"""
import pathlib

import numpy as np

GOLDEN = pathlib.Path(__file__).parent / "golden"
VARS = ("u", "v", "sxx", "syy", "sxy")


def load_table1():
    rows = []
    for line in (GOLDEN / "table1_convergence.txt").read_text().splitlines():
        if not line.strip() or line.lstrip().startswith("#"):
            continue
        f = line.split()
        p, n = int(f[0]), int(f[1])
        err = np.array([float(f[2 + 2 * k]) for k in range(5)])
        rate = np.array([np.nan if f[3 + 2 * k] == "-" else float(f[3 + 2 * k]) for k in range(5)])
        rows.append(dict(p=p, n=n, err=err, rate=rate, t_cpu=float(f[12])))
    return rows


def load_sliver():
    out = {}
    for line in (GOLDEN / "sliver_iterations.txt").read_text().splitlines():
        if not line.strip() or line.lstrip().startswith("#"):
            continue
        name, m1, m2, fac = line.split()
        out[name] = (float(m1), float(m2), float(fac))
    return out


def test_table1_rates_follow_the_mesh_size_reading():
    rows = load_table1()
    assert sorted({r["p"] for r in rows}) == [1, 2, 3, 4]
    ns = [r["n"] for r in rows if r["p"] == 1]
    assert ns == [1760, 3960, 7040, 11000]
    h = 0.1264 * np.sqrt(1760.0 / np.array(ns))
    assert np.allclose(h, [0.1264, 0.0842, 0.0632, 0.0505], atol=1e-4)   # the paper truncates
    garbled = np.array([0.1264, 0.0842, 0.0842, 0.0505])
    worst_garbled = 0.0
    for p in (1, 2, 3, 4):
        rs = [r for r in rows if r["p"] == p]
        assert [r["n"] for r in rs] == ns
        for k in range(1, 4):
            e0, e1 = rs[k - 1]["err"], rs[k]["err"]
            rate = np.log(e0 / e1) / np.log(h[k - 1] / h[k])
            assert np.all(np.abs(rate - rs[k]["rate"]) <= 0.051), (p, k, rate, rs[k]["rate"])
            with np.errstate(divide="ignore"):
                g = np.log(e0 / e1) / np.log(garbled[k - 1] / garbled[k])
            worst_garbled = max(worst_garbled, float(np.max(np.abs(g - rs[k]["rate"]))))
    assert worst_garbled > 1.0


def test_table1_finest_rates_reach_p_plus_one():
    for r in load_table1():
        if r["n"] == 11000:
            assert np.all(r["rate"] >= r["p"] + 1 - 0.05), (r["p"], r["rate"])
            # the errors themselves fall with p on every mesh of the table
    rows = load_table1()
    for n in (1760, 3960, 7040, 11000):
        e = [r["err"] for r in sorted(rows, key=lambda r: r["p"]) if r["n"] == n]
        assert all(np.all(e[i + 1] < e[i]) for i in range(3))


def test_sliver_table_ordering():
    t = load_sliver()
    assert set(t) == {"none", "pre1", "pre2"}
    for m1, m2, fac in t.values():
        assert abs(m2 / m1 - fac) <= 0.01   # printed to two decimals, truncated
    for k in (0, 1):
        assert t["none"][k] > t["pre1"][k] > t["pre2"][k]
    assert t["none"][2] > t["pre1"][2] > t["pre2"][2]
    assert abs(t["pre2"][2] - 1.0) < 0.01
