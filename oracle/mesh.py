"""Element and surface quantities of a tetrahedral mesh (Sec. II-A, Eq. 1).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

# Centering operator N = I_4 - (1/4) 1 1^T of Eq. 1.  The paper prints N V with
# V of size 3x4; the product that is defined is V N (column centering).
N4 = np.eye(4) - 0.25 * np.ones((4, 4))

# Outward faces of a positively oriented tet (v0, v1, v2, v3): face k is the
# face opposite local vertex k, listed counter-clockwise seen from outside.
TET_FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))


def element_matrices(X: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """V_e in R^{3x4} for every tet: columns are the 4 vertex positions."""
    return X[tets].transpose(0, 2, 1).copy()


def centered(V: np.ndarray) -> np.ndarray:
    """V N (Eq. 1): subtract the element centroid from each column."""
    return V @ N4


def signed_volume(V: np.ndarray) -> np.ndarray:
    """Vol of a 3x4 element: det[v1-v0, v2-v0, v3-v0] / 6 (positive for the
    orientation used throughout)."""
    E = V[:, :, 1:] - V[:, :, :1]
    return np.linalg.det(E) / 6.0


def rest_quantities(rest: np.ndarray, tets: np.ndarray):
    """Rest centered shapes T_c = V_rest N, rest volumes and element weights.

    The paper weights elements by Vol(e) in Eq. 1 and by omega_e in Eq. 8; this
    oracle uses omega_e = Vol(e) / mean Vol, the same weighting up to a global
    scale, which equals 1 on uniform Kuhn meshes."""
    V = element_matrices(rest, tets)
    T_c = centered(V)
    vol0 = signed_volume(V)
    omega = vol0 / vol0.mean()
    return T_c, vol0, omega


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one tet, as (n_f, 3) vertex triples,
    oriented outward, ordered by (tet id, local face index)."""
    n_t = tets.shape[0]
    tri = np.stack([tets[:, list(f)] for f in TET_FACES], axis=1)      # (n_t, 4, 3)
    keys = np.sort(tri.reshape(-1, 3), axis=1)
    _, inv, counts = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
    once = counts[inv.ravel()] == 1
    order = np.arange(n_t * 4)
    return tri.reshape(-1, 3)[order[once]]


def surface_vertices(faces: np.ndarray) -> np.ndarray:
    """Sorted vertex ids that lie on a boundary face."""
    return np.unique(faces.ravel())


def face_normals(X: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """Unnormalised outward face normals (q1 - q0) x (q2 - q0)."""
    q0, q1, q2 = X[faces[:, 0]], X[faces[:, 1]], X[faces[:, 2]]
    return np.cross(q1 - q0, q2 - q0)


def vertex_normals(X: np.ndarray, faces: np.ndarray, n_verts: int) -> np.ndarray:
    """Area-weighted vertex normals: the normalised sum of the unnormalised
    normals of the incident boundary faces (zero for interior vertices)."""
    fn = face_normals(X, faces)
    acc = np.zeros((n_verts, 3))
    for k in range(3):
        np.add.at(acc, faces[:, k], fn)
    nrm = np.linalg.norm(acc, axis=1)
    out = np.zeros_like(acc)
    nz = nrm > 0
    out[nz] = acc[nz] / nrm[nz, None]
    return out
