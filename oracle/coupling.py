"""CPU FP64 oracle for the sparse coupling blocks of the hybrid system (Eq. 42).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package.  It shares
no code with the CUDA path.

  D^{J Lambda}_mn = -<j_m, (1/2) n x eta_n>_{T_m}        Eq. 47
  D^{M Lambda}_mn =  <m_m, (1/2) pi^tau eta_n>_{T_m}     Eq. 48
  D^{Lambda J}_mn = -<eta_m, n x j_n>                     Eq. 40a
  D^{Lambda M}_mn = -<eta_m, pi^tau m_n>                  Eq. 40b

j, m are the RWG functions of the surface (Sec. II.D, Eq. exp4-5, in the order and sign of
oracle.rwg); eta are the 2-D zeroth-order vector edge functions of Eq. exp3 on the surface
triangles.  Readings: eta is tangential on its triangle, so pi^tau eta = eta and
pi^tau m = m; n is the outward unit normal of the triangle; the edge function of the edge
(a, b) of a triangle, a the smaller global vertex number, is
    eta = l_ab (lambda_a grad lambda_b - lambda_b grad lambda_a)
(lambda the barycentric coordinates, l_ab the edge length), so that its tangential component
along the edge, from a to b, is 1.  Two layouts of the Lambda unknowns:
  conforming=False: one function per (triangle, local edge k), index 3 t + k, k the edge
                    opposite local vertex k: the face-wise space of a hybridised method;
  conforming=True:  one function per mesh edge, in the RWG order, the sum of the two
                    face functions of that edge (tangentially continuous across it).
Each integral is a product of two linear functions on a flat triangle, so the three-point
edge-midpoint rule (weights A/3) integrates it exactly.
"""
import numpy as np

from . import rwg as _rwg

# barycentric coordinates of the edge midpoints: point q is the midpoint of the edge
# opposite local vertex q
_LAM = np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def face_frame(P):
    """Area, unit normal and barycentric gradients of the triangle with vertex rows P [3][3].
    The gradients come from the pseudo-inverse of the edge matrix [P1 - P0, P2 - P0]."""
    P = np.asarray(P, np.float64)
    E = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)           # 3 x 2
    c = np.cross(E[:, 0], E[:, 1])
    A = 0.5 * np.linalg.norm(c)
    g12 = np.linalg.pinv(E)                                      # rows: grad lambda_1, grad lambda_2
    grads = np.stack([-g12[0] - g12[1], g12[0], g12[1]])
    return A, c / np.linalg.norm(c), grads


def whitney(P, gid, k, lam):
    """Edge function of the edge opposite local vertex k of the triangle P (global vertex
    numbers gid[3]) at the points with barycentric coordinates lam [npts][3]."""
    _, _, grads = face_frame(P)
    a, b = (k + 1) % 3, (k + 2) % 3
    if gid[a] > gid[b]:
        a, b = b, a
    lab = np.linalg.norm(P[b] - P[a])
    lam = np.atleast_2d(lam)
    return lab * (lam[:, [a]] * grads[b][None, :] - lam[:, [b]] * grads[a][None, :])


def rwg_on_face(P, free, length, sign, lam):
    """RWG function at barycentric points lam of its triangle P: sign * l / (2A) * (r - p),
    p the free vertex (local index `free`), sign +1 on T+ and -1 on T-."""
    A, _, _ = face_frame(P)
    r = np.atleast_2d(lam) @ P
    return sign * length / (2 * A) * (r - P[free][None, :])


def coupling_blocks(verts, tris, conforming=False):
    """Dense (D^{J Lambda}, D^{M Lambda}, D^{Lambda J}, D^{Lambda M}) as float64 arrays of
    shapes [N][nL], [N][nL], [nL][N], [nL][N] (N RWG functions, nL Lambda functions)."""
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64)
    R = _rwg(v, t)
    N, nt = len(R["edges"]), len(t)
    edge_id = {}
    for n, (a, b) in enumerate(R["edges"]):
        edge_id[(int(a), int(b))] = n
    nL = N if conforming else 3 * nt
    DJL = np.zeros((N, nL))
    DML = np.zeros((N, nL))
    DLJ = np.zeros((nL, N))
    DLM = np.zeros((nL, N))
    on_face = [[] for _ in range(nt)]                            # (rwg, free local vertex, sign)
    for n in range(N):
        on_face[R["tplus"][n]].append((n, int(R["lplus"][n]), 1.0))
        on_face[R["tminus"][n]].append((n, int(R["lminus"][n]), -1.0))
    for f in range(nt):
        P = v[t[f]]
        A, nrm, _ = face_frame(P)
        w = A / 3.0
        for k in range(3):
            eta = whitney(P, t[f], k, _LAM)
            n_eta = np.cross(nrm[None, :], eta)
            if conforming:
                ga, gb = sorted((int(t[f][(k + 1) % 3]), int(t[f][(k + 2) % 3])))
                col = edge_id[(ga, gb)]
            else:
                col = 3 * f + k
            for m, free, s in on_face[f]:
                a, b = R["edges"][m]
                fm = rwg_on_face(P, free, np.linalg.norm(v[b] - v[a]), s, _LAM)
                n_fm = np.cross(nrm[None, :], fm)
                DJL[m, col] += -0.5 * w * np.sum(fm * n_eta)
                DML[m, col] += 0.5 * w * np.sum(fm * eta)
                DLJ[col, m] += -w * np.sum(eta * n_fm)
                DLM[col, m] += -w * np.sum(eta * fm)
    return DJL, DML, DLJ, DLM


def coupling_matrices(verts, tris, conforming=False):
    """The blocks arranged as in Eq. 42 for the unknowns [J; M]: D^{X Lambda} = [D^{J Lambda};
    D^{M Lambda}] ([2N][nL]) and D^{Lambda X} = [D^{Lambda J}, D^{Lambda M}] ([nL][2N])."""
    DJL, DML, DLJ, DLM = coupling_blocks(verts, tris, conforming)
    return np.vstack([DJL, DML]), np.hstack([DLJ, DLM])
