"""The C ABI from plain C99 (no C++, no Python): a client that includes include/stdg.h
compiles with gcc -std=c99 -Wall -Werror, links libstdg.so and calls the context-free
functions (face table, point location, reference tables); its output is checked against
the oracle.  CPU only: these calls touch no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.mesh import DualMesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CLIENT = r"""
#include <stdio.h>
#include <stdlib.h>
#include "stdg.h"

int main(void) {
    /* mesh read from stdin: n_vert n_elem, coordinates, vertex ids; period 1 x 1 */
    long long nv, ne;
    if (scanf("%lld %lld", &nv, &ne) != 2) return 2;
    double* xyz = malloc(sizeof(double) * 2 * nv);
    int32_t* ev = malloc(sizeof(int32_t) * 3 * ne);
    for (long long i = 0; i < 2 * nv; ++i) if (scanf("%lf", &xyz[i]) != 1) return 2;
    for (long long i = 0; i < 3 * ne; ++i) if (scanf("%d", &ev[i]) != 1) return 2;
    double period[2] = {1.0, 1.0};
    int64_t nf = 0;
    int rc = stdg_mesh_faces(2, nv, xyz, ne, ev, period, &nf, NULL, NULL);
    if (rc != STDG_OK) return 3;
    int32_t* fl = malloc(sizeof(int32_t) * nf);
    int32_t* fr = malloc(sizeof(int32_t) * nf);
    rc = stdg_mesh_faces(2, nv, xyz, ne, ev, period, &nf, fl, fr);
    if (rc != STDG_OK) return 4;
    printf("faces %lld\n", (long long)nf);
    for (int64_t j = 0; j < nf; ++j) printf("%d %d\n", fl[j], fr[j]);
    double pts[4] = {0.31, 0.62, 0.77, 0.05};
    int64_t el[2];
    rc = stdg_locate_points(2, nv, xyz, ne, ev, period, 2, pts, el);
    if (rc != STDG_OK) return 5;
    printf("located %lld %lld\n", (long long)el[0], (long long)el[1]);
    double W[2], kappa;
    rc = stdg_reference_tables(2, 1, 1, NULL, W, NULL, NULL, &kappa, NULL);
    if (rc != STDG_OK) return 6;
    printf("tables %.17g %.17g %.17g\n", W[0], W[1], kappa);
    printf("null %d\n", stdg_step(NULL, 0.1, 1, NULL));
    free(xyz); free(ev); free(fl); free(fr);
    return 0;
}
"""


def test_plain_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1802_04516_gb300 import build
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-lstdg", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    xyz, ev, per = synth.tri_grid(4, 3, 1.0, 1.0, periodic=True, jitter=0.2, seed=4)
    feed = "%d %d\n" % (len(xyz), len(ev)) + " ".join("%.17g" % v for v in xyz.ravel()) + "\n" + \
        " ".join(str(int(v)) for v in ev.ravel()) + "\n"
    r = subprocess.run([str(exe)], input=feed, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = r.stdout.splitlines()
    m = DualMesh(xyz, ev, per)
    nf = int(lines[0].split()[1])
    assert nf == m.n_face
    table = np.array([[int(a) for a in ln.split()] for ln in lines[1:1 + nf]])
    assert np.array_equal(table[:, 0], m.face_l) and np.array_equal(table[:, 1], m.face_r)
    loc = [int(a) for a in lines[1 + nf].split()[1:]]
    assert loc == [m.locate(np.array([0.31, 0.62]))[0], m.locate(np.array([0.77, 0.05]))[0]]
    W0, W1, kappa = (float(a) for a in lines[2 + nf].split()[1:])
    from oracle.basis import TimeBasis
    tm = TimeBasis(1).matrices()
    assert abs(W0 - 0.5) < 1e-15 and abs(W1 - 0.5) < 1e-15
    assert abs(kappa - tm["g1"] @ np.linalg.solve(tm["T"], tm["g0"])) < 1e-13
    assert lines[3 + nf] == "null -1"
