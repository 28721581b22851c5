"""Independent closed forms and dense brute force used to pin the oracle.

Nothing here calls the oracle's element routines: bricks use the exact tensor-product
integrals of 1-D linear shape functions, tetrahedra use face area vectors, and assembly is a
dense global matrix.  These are textbook identities, not the oracle's quadrature code.
"""
import numpy as np

# VTK hex node -> (ix, iy, iz) corner indices
VTK_CORNERS = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                        (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)])


def _m1(h):   # int N_i N_j on [0,h]
    return h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])


def _s1(h):   # int N_i' N_j'
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def _g1(h):   # int N_i' N_j
    return np.array([[-0.5, -0.5], [0.5, 0.5]])


def brick_K(dims, k):
    """Exact conduction matrix of the rectangular brick [0,a]x[0,b]x[0,c] (VTK order) with a
    constant 3x3 conductivity k: K_ij = sum_ab k_ab int d_a N_i d_b N_j as products of 1-D
    integrals."""
    k = np.asarray(k, float)
    M = [_m1(h) for h in dims]
    S = [_s1(h) for h in dims]
    G = [_g1(h) for h in dims]
    K = np.zeros((8, 8))
    for i in range(8):
        ci = VTK_CORNERS[i]
        for j in range(8):
            cj = VTK_CORNERS[j]
            tot = 0.0
            for a in range(3):
                for b in range(3):
                    f = 1.0
                    for ax in range(3):
                        if a == b == ax:
                            f *= S[ax][ci[ax], cj[ax]]
                        elif ax == a and a != b:
                            f *= G[ax][ci[ax], cj[ax]]
                        elif ax == b and a != b:
                            f *= G[ax][cj[ax], ci[ax]]
                        else:
                            f *= M[ax][ci[ax], cj[ax]]
                    tot += k[a, b] * f
            K[i, j] = tot
    return K


def tet_K_facevec(x, k):
    """Linear-tet conduction matrix from outward face area vectors S_i (face opposite node i):
    grad N_i = -S_i / (3V), so K_ij = S_i . k S_j / (9 V)."""
    x = np.asarray(x, float)
    V = np.dot(np.cross(x[1] - x[0], x[2] - x[0]), x[3] - x[0]) / 6.0
    S = np.zeros((4, 3))
    for i in range(4):
        j, l, m = [q for q in range(4) if q != i]
        n = 0.5 * np.cross(x[l] - x[j], x[m] - x[j])
        if np.dot(n, x[j] - x[i]) < 0:
            n = -n
        S[i] = n
    return S @ np.asarray(k, float) @ S.T / (9.0 * V), V


def dense_assemble(conn, Ke, nn, scale=None):
    """Global K = sum_e scale_e K_e, assembled densely."""
    K = np.zeros((nn, nn))
    for e, c in enumerate(conn):
        s = 1.0 if scale is None else scale[e]
        K[np.ix_(c, c)] += s * Ke[e]
    return K


def c1_closed_form(n, dt, nsteps, T0=100.0):
    """Fully discrete solution of the plain cube (unit cube, n^3 bricks, k = rho = c = 1,
    T = 0 on the boundary, T0 inside) after nsteps forward-Euler steps with lumped mass: the
    sine vectors diagonalise both the assembled brick K and the lumped mass h^3.  Returns the
    nodal field on the full (n+1)^3 grid (node id = i + (n+1)(j + (n+1)k))."""
    h = 1.0 / n
    idx = np.arange(1, n)
    l = np.arange(1, n)
    Sx = np.sin(np.pi * np.outer(l, idx) * h)            # [mode, node]
    kap = (2.0 / h) * (1.0 - np.cos(l * np.pi * h))
    mu = (h / 3.0) * (2.0 + np.cos(l * np.pi * h))
    # DST-I coefficients of the interior initial field (orthogonality: sum sin^2 = n/2)
    a = np.full((n - 1,) * 3, T0)
    a = np.einsum("li,mj,pk,kji->pml", Sx, Sx, Sx, a) * (2.0 / n) ** 3   # index [p,m,l]
    lam = (kap[None, None, :] * mu[None, :, None] * mu[:, None, None]
           + mu[None, None, :] * kap[None, :, None] * mu[:, None, None]
           + mu[None, None, :] * mu[None, :, None] * kap[:, None, None]) / h ** 3
    coef = a * (1.0 - dt * lam) ** nsteps
    inner = np.einsum("pml,li,mj,pk->kji", coef, Sx, Sx, Sx)            # [k,j,i]
    T = np.zeros((n + 1,) * 3)
    T[1:n, 1:n, 1:n] = inner
    return T.reshape(-1), lam.max()


def ftcs_slab(nx, h, dt, nsteps, T0, Ts, k, rho, c0, k_lin=0.0, c_lin=0.0, conv=None,
              source=0.0, Ts_offset=None, fk_fn=None, fc_fn=None):
    """1-D forward-Euler recurrence equivalent to a bar of bricks whose field is constant over
    each cross-section (consistent row sums = lumped mass):
      interior  T_j += dt k / (rho c(T_j) h^2) [f_R (T_{j+1}-T_j) + f_L (T_{j-1}-T_j)]
      x = L end T_n += 2 dt k / (rho c(T_n) h^2) f_L (T_{n-1}-T_n) - 2 dt hc/(rho c(T_n) h) (T_n - T_inf)
    with f on an element = 1 + k_lin (T_left + T_right)/2 and c(T) = c0 (1 + c_lin T); a
    uniform volumetric source s adds dt s / (rho c(T_j)) to every free node.  With Ts_offset
    the held end is Ts + Ts_offset[n] at step n (the last entry beyond the end).  With fk_fn /
    fc_fn (callables of the nodal temperature) the element factor is the mean of fk_fn over
    its two end temperatures and c(T) = c0 fc_fn(T)."""
    def end_value(n):
        if Ts_offset is None:
            return Ts
        return Ts + Ts_offset[min(n, len(Ts_offset) - 1)]

    T = np.full(nx + 1, float(T0))
    T[0] = end_value(0)
    for n in range(nsteps):
        if fk_fn is None:
            f = 1.0 + k_lin * 0.5 * (T[:-1] + T[1:])      # per element
        else:
            fn = fk_fn(T)
            f = 0.5 * (fn[:-1] + fn[1:])
        c = c0 * (1.0 + c_lin * T) if fc_fn is None else c0 * fc_fn(T)
        Tn = T.copy()
        Tn[1:-1] = T[1:-1] + dt * k / (rho * c[1:-1] * h * h) * (
            f[1:] * (T[2:] - T[1:-1]) + f[:-1] * (T[:-2] - T[1:-1]))
        Tn[-1] = T[-1] + 2.0 * dt * k / (rho * c[-1] * h * h) * f[-1] * (T[-2] - T[-1])
        if conv is not None:
            hc, Tinf = conv
            Tn[-1] -= 2.0 * dt * hc / (rho * c[-1] * h) * (T[-1] - Tinf)
        Tn[1:] += dt * source / (rho * c[1:])
        Tn[0] = end_value(n + 1)
        T = Tn
    return T
