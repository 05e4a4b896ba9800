"""Primary mesh, faces and face-based dual cells (Sec. 3, "Two space dimensions",
"Three space dimensions").

Readings of what the paper leaves open (the library implements the same ones):
  * l(j), r(j) are "assigned arbitrarily": here l(j) is the smaller element index,
    r(j) the larger; n_j is the unit normal of Gamma_j pointing from l(j) to r(j),
    and outward of l(j) on a boundary face.
  * the sign s_{i,j} of Eq. SD_1 is +1 for i = l(j), -1 for i = r(j); a mesh in
    which an element is its own neighbour (l = r, a periodic direction one cell
    wide) is rejected.
  * faces are numbered in ascending lexicographic order of their sorted global
    vertex-id tuple; local face f of an element is the one opposite its vertex f.
  * on a periodic axis the dual cell that straddles the seam is unwrapped into the
    frame of l(j): r(j)'s coordinates are shifted by whole periods.
  * a boundary face (free surface) has the single sub-cell T_{l,j}.
  * sub-cell T_{i,j} = simplex(face vertices, barycenter of T_i); the dual-cell
    "centre" x_j is the measure-weighted centroid of R_j and h_j the largest
    distance from x_j to a vertex of R_j (these fix the Taylor dual basis).
Pins: Theorem 1 symmetry / Q~ = -D^T and the constant-stress identity, which fail
for a wrong normal orientation or frame shift (tests/test_oracle_operators.py).
"""
import numpy as np


def _unwrap(xyz, elem, period):
    X = xyz[elem].astype(np.float64)
    if period is not None:
        for a in range(X.shape[2]):
            L = float(period[a])
            if L > 0:
                X[:, :, a] -= L * np.round((X[:, :, a] - X[:, :1, a]) / L)
    return X


def _det(E):
    return np.linalg.det(E)


class DualMesh:
    def __init__(self, xyz, elem_vert, period=None):
        elem = np.asarray(elem_vert, dtype=np.int64)
        self.dim = d = elem.shape[1] - 1
        self.n_elem = elem.shape[0]
        self.elem = elem
        self.period = None if period is None else np.asarray(period, dtype=np.float64)
        X = _unwrap(np.asarray(xyz, dtype=np.float64), elem, self.period)
        self.X = X
        J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # columns = edges
        detJ = _det(J)
        if (detJ <= 0).any():
            raise ValueError("inverted or degenerate element")
        self.J = J
        self.detJ = detJ
        self.Jinv = np.linalg.inv(J)
        self.vol = detJ / (2.0 if d == 2 else 6.0)
        self.bary = X.mean(axis=1)

        # faces by sorted global vertex tuple
        table = {}
        for i in range(self.n_elem):
            for f in range(d + 1):
                key = tuple(sorted(int(v) for k, v in enumerate(elem[i]) if k != f))
                table.setdefault(key, []).append((i, f))
        keys = sorted(table)
        nf = len(keys)
        self.n_face = nf
        self.face_l = np.zeros(nf, dtype=np.int64)
        self.face_r = np.full(nf, -1, dtype=np.int64)
        self.face_fl = np.zeros(nf, dtype=np.int64)
        self.face_fr = np.full(nf, -1, dtype=np.int64)
        self.elem_faces = np.zeros((self.n_elem, d + 1), dtype=np.int64)
        self.elem_nbr = np.full((self.n_elem, d + 1), -1, dtype=np.int64)
        for j, key in enumerate(keys):
            ent = sorted(table[key])
            if len(ent) > 2:
                raise ValueError("non-manifold face")
            if len(ent) == 2 and ent[0][0] == ent[1][0]:
                raise ValueError("element is its own neighbour")
            (il, fl) = ent[0]
            self.face_l[j], self.face_fl[j] = il, fl
            self.elem_faces[il, fl] = j
            if len(ent) == 2:
                (ir, fr) = ent[1]
                self.face_r[j], self.face_fr[j] = ir, fr
                self.elem_faces[ir, fr] = j
                self.elem_nbr[il, fl] = ir
                self.elem_nbr[ir, fr] = il
        self.interior = self.face_r >= 0

        # face geometry in the frame of l(j)
        self.face_X = np.zeros((nf, d, d))      # face vertices (l frame, l's local order)
        self.shift = np.zeros((nf, d))          # add to r-frame coordinates -> l frame
        for j in range(nf):
            il, fl = self.face_l[j], self.face_fl[j]
            loc = [k for k in range(d + 1) if k != fl]
            self.face_X[j] = X[il, loc]
            if self.face_r[j] >= 0:
                ir = self.face_r[j]
                g = elem[il, loc[0]]
                kr = int(np.where(elem[ir] == g)[0][0])
                self.shift[j] = X[il, loc[0]] - X[ir, kr]
        self.normal = np.zeros((nf, d))
        self.area = np.zeros(nf)
        for j in range(nf):
            F = self.face_X[j]
            if d == 2:
                t = F[1] - F[0]
                n = np.array([t[1], -t[0]])
                self.area[j] = np.linalg.norm(t)
            else:
                n = np.cross(F[1] - F[0], F[2] - F[0])
                self.area[j] = 0.5 * np.linalg.norm(n)
            n = n / np.linalg.norm(n)
            opp = X[self.face_l[j], self.face_fl[j]]
            if np.dot(n, F[0] - opp) < 0:
                n = -n
            self.normal[j] = n

        # dual cells R_j: centre x_j and scale h_j (l frame)
        self.sub_vol = self.vol / (d + 1)
        self.xc = np.zeros((nf, d))
        self.hj = np.zeros(nf)
        for j in range(nf):
            il = self.face_l[j]
            F = self.face_X[j]
            pts = [F[k] for k in range(d)] + [self.bary[il]]
            cen = (F.sum(axis=0) + self.bary[il]) / (d + 1)
            m = self.sub_vol[il]
            num = m * cen
            den = m
            if self.face_r[j] >= 0:
                ir = self.face_r[j]
                br = self.bary[ir] + self.shift[j]
                pts.append(br)
                cen_r = (F.sum(axis=0) + br) / (d + 1)
                num = num + self.sub_vol[ir] * cen_r
                den = den + self.sub_vol[ir]
            self.xc[j] = num / den
            self.hj[j] = max(np.linalg.norm(q - self.xc[j]) for q in pts)

    # --- pairs (i, j) with j in S_i -------------------------------------------------
    def pairs(self):
        """List of (element, face, side) with side 0 = l(j), 1 = r(j)."""
        out = [(int(self.face_l[j]), j, 0) for j in range(self.n_face)]
        out += [(int(self.face_r[j]), j, 1) for j in range(self.n_face) if self.face_r[j] >= 0]
        return out

    def face_vertices_in_frame(self, j, side):
        """Face vertices in the frame of element l(j) (side 0) or r(j) (side 1)."""
        return self.face_X[j] if side == 0 else self.face_X[j] - self.shift[j]

    def locate(self, x, tol=1e-12):
        """Element containing point x (lowest index wins) and x in that element's frame."""
        x = np.asarray(x, dtype=np.float64)
        for i in range(self.n_elem):
            y = x.copy()
            if self.period is not None:
                for a in range(self.dim):
                    L = self.period[a]
                    if L > 0:
                        y[a] -= L * np.round((y[a] - self.X[i, 0, a]) / L)
            xi = self.Jinv[i] @ (y - self.X[i, 0])
            lam = np.concatenate([[1.0 - xi.sum()], xi])
            if (lam >= -tol).all():
                return i, y
        raise ValueError("point outside the mesh")
