"""Test helpers: dense reconstructions from exported arrays (numpy only)."""
import numpy as np


def dense_from_bsr(rp, ci, blocks, d):
    n = (len(rp) - 1) * d
    A = np.zeros((n, n))
    for i in range(len(rp) - 1):
        for k in range(rp[i], rp[i + 1]):
            j = ci[k]
            A[i * d:(i + 1) * d, j * d:(j + 1) * d] = blocks[k]
    return A


def dense_P(rp, ci, w, n_coarse, d, dead_fine=None):
    """Dof-level prolongation P_s (x) I_d with rows of dead fine dofs zeroed."""
    nf = len(rp) - 1
    P = np.zeros((nf * d, n_coarse * d))
    for i in range(nf):
        for k in range(rp[i], rp[i + 1]):
            for c in range(d):
                if dead_fine is None or not dead_fine[i * d + c]:
                    P[i * d + c, ci[k] * d + c] = w[k]
    return P


def deinterleave(keys, d, bits):
    keys = np.asarray(keys, dtype=np.uint64)
    out = np.zeros((keys.size, d), dtype=np.uint64)
    for b in range(bits):
        for a in range(d):
            out[:, a] |= ((keys >> np.uint64(b * d + a)) & np.uint64(1)) << np.uint64(b)
    return out


def interleave(coords, d, bits):
    coords = np.asarray(coords, dtype=np.uint64)
    k = np.zeros(coords.shape[0], dtype=np.uint64)
    for b in range(bits):
        for a in range(d):
            k |= ((coords[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(b * d + a)
    return k


def K_of(d):
    return 31 if d == 2 else 20


def rigid_modes(coords):
    """Translations and infinitesimal rotations of the point set (dof-major rows)."""
    nv, d = coords.shape
    modes = []
    for a in range(d):
        t = np.zeros((nv, d))
        t[:, a] = 1.0
        modes.append(t.ravel())
    x = coords - coords.mean(axis=0)
    if d == 2:
        r = np.zeros((nv, 2))
        r[:, 0] = -x[:, 1]
        r[:, 1] = x[:, 0]
        modes.append(r.ravel())
    else:
        for (a, b) in [(0, 1), (1, 2), (0, 2)]:
            r = np.zeros((nv, 3))
            r[:, a] = -x[:, b]
            r[:, b] = x[:, a]
            modes.append(r.ravel())
    return modes


def voigt_element_stiffness(X, lam, mu):
    """Element stiffness |K| B^T D B in Voigt notation (textbook form, independent
    of the paper's block form).  X: (d+1, d) vertex coordinates.  Returns a
    ((d+1)d, (d+1)d) matrix in vertex-interleaved dof order."""
    d = X.shape[1]
    J = (X[1:] - X[0]).T  # J[a, k] = x_{k+1,a} - x_{0,a}
    G = np.linalg.inv(J)  # rows: gradients of basis 1..d
    grads = np.vstack([-G.sum(axis=0), G])
    meas = abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)
    nl = d + 1
    if d == 2:
        B = np.zeros((3, 2 * nl))
        for k in range(nl):
            gx, gy = grads[k]
            B[0, 2 * k] = gx
            B[1, 2 * k + 1] = gy
            B[2, 2 * k] = gy
            B[2, 2 * k + 1] = gx
        D = np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
    else:
        B = np.zeros((6, 3 * nl))
        for k in range(nl):
            gx, gy, gz = grads[k]
            B[0, 3 * k] = gx
            B[1, 3 * k + 1] = gy
            B[2, 3 * k + 2] = gz
            B[3, 3 * k] = gy
            B[3, 3 * k + 1] = gx
            B[4, 3 * k + 1] = gz
            B[4, 3 * k + 2] = gy
            B[5, 3 * k] = gz
            B[5, 3 * k + 2] = gx
        D = np.zeros((6, 6))
        D[:3, :3] = lam
        D[[0, 1, 2], [0, 1, 2]] = lam + 2 * mu
        D[[3, 4, 5], [3, 4, 5]] = mu
    return meas * B.T @ D @ B
