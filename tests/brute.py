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


def hex_shape_integrals_gauss3(x):
    """w_i = int_Ve N_i dV of a trilinear hexahedron (VTK order) by 3x3x3 Gauss-Legendre points
    (numpy's leggauss), with the shape functions written as products of 1-D linear functions
    of the corner index bits.  N_i det J has degree <= 3 in each natural coordinate, so both
    this rule (exact to degree 5) and the 2x2x2 rule (exact to degree 3) integrate it exactly;
    the two share no code.  Returns (w [8], volume)."""
    x = np.asarray(x, float)
    g, gw = np.polynomial.legendre.leggauss(3)
    sgn = 2.0 * VTK_CORNERS - 1.0                      # [8, 3] corner signs
    w = np.zeros(8)
    vol = 0.0
    for a, wa in zip(g, gw):
        for b, wb in zip(g, gw):
            for c, wc in zip(g, gw):
                p = np.array([a, b, c])
                lin = 0.5 * (1.0 + sgn * p)             # [8, 3] 1-D factors
                N = np.prod(lin, axis=1)
                dN = np.empty((8, 3))
                for d in range(3):
                    o = [q for q in range(3) if q != d]
                    dN[:, d] = 0.5 * sgn[:, d] * lin[:, o[0]] * lin[:, o[1]]
                J = x.T @ dN                            # dx_r / dxi_s
                dj = np.linalg.det(J)
                w += wa * wb * wc * dj * N
                vol += wa * wb * wc * dj
    return w, vol


def hex_shape_integrals_exact(x):
    """Exact w_i = int N_i det J over [-1,1]^3 as a polynomial integral in rational arithmetic
    (sympy), for coordinates given as decimals.  Returns (w [8] as floats, volume)."""
    import sympy as sp
    xi = sp.symbols("xi0:3")
    X = [[sp.Rational(str(float(v))) for v in row] for row in np.asarray(x, float)]
    N = []
    for ci in VTK_CORNERS:
        f = sp.Integer(1)
        for d in range(3):
            f *= (1 + (2 * int(ci[d]) - 1) * xi[d]) / 2
        N.append(sp.expand(f))
    J = sp.Matrix(3, 3, lambda r, s: sum(X[i][r] * sp.diff(N[i], xi[s]) for i in range(8)))
    dj = sp.expand(J.det())

    def integ(f):
        for v in xi:
            f = sp.integrate(f, (v, -1, 1))
        return f
    w = [integ(sp.expand(Ni * dj)) for Ni in N]
    return np.array([float(v) for v in w]), float(integ(dj))


def hex_load_exact_qp(x, k, T, fk, order=3):
    """F_i = int_Ve grad N_i . k fk(T(x)) grad T dV on a trilinear hexahedron (VTK order) for the
    nodal field T, by 3x3x3 Gauss-Legendre points with shape functions written as products of
    1-D linear functions: exact on rectangular bricks when fk is linear (the integrand then has
    degree <= 3 per coordinate).  fk: callable of the temperature; order: Gauss points per
    direction (order = 2 applies the 2x2x2 rule itself, for distorted elements)."""
    x = np.asarray(x, float)
    T = np.asarray(T, float)
    k = np.asarray(k, float)
    g, gw = np.polynomial.legendre.leggauss(order)
    sgn = 2.0 * VTK_CORNERS - 1.0
    F = np.zeros(8)
    for a, wa in zip(g, gw):
        for b, wb in zip(g, gw):
            for c, wc in zip(g, gw):
                p = np.array([a, b, c])
                lin = 0.5 * (1.0 + sgn * p)
                N = np.prod(lin, axis=1)
                dN = np.empty((8, 3))
                for d in range(3):
                    o = [q for q in range(3) if q != d]
                    dN[:, d] = 0.5 * sgn[:, d] * lin[:, o[0]] * lin[:, o[1]]
                J = x.T @ dN
                B = dN @ np.linalg.inv(J)          # [8, 3] physical gradients
                gradT = B.T @ T
                F += wa * wb * wc * np.linalg.det(J) * fk(N @ T) * (B @ (k @ gradT))
    return F


def bar_lateral_convection(nx, h, w, dt, nsteps, T0, Ts, k, rho, c0, hc, Tinf, consistent):
    """Forward-Euler recurrence of a bar of nx bricks (h along x, cross-section w x w), T = Ts
    held at x = 0, convection hc (T - Tinf) on the four lateral faces, for fields constant over
    each cross-section.  Per node (lumped brick mass rho c0 w^2 h / 4 inside, half at the end):
      conduction  k w^2 / (4 h) (T_{j-1} - 2 T_j + T_{j+1})
      lumped      -hc w h T'_j                        (T' = T - Tinf; area share w h / 4 per face)
      consistent  -(hc w h / 6)(T'_{j-1} + 4 T'_j + T'_{j+1}), end node -(hc w h / 6)(2 T'_n + T'_{n-1})
    from the bilinear face mass matrix (w h / 36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4]."""
    T = np.full(nx + 1, float(T0))
    T[0] = Ts
    m_in = rho * c0 * w * w * h / 4.0
    for _ in range(nsteps):
        Tp = T - Tinf
        cond = np.zeros(nx + 1)
        cond[1:-1] = k * w * w / (4.0 * h) * (T[:-2] - 2.0 * T[1:-1] + T[2:])
        cond[-1] = k * w * w / (4.0 * h) * (T[-2] - T[-1])
        if consistent:
            conv = np.zeros(nx + 1)
            conv[1:-1] = -(hc * w * h / 6.0) * (Tp[:-2] + 4.0 * Tp[1:-1] + Tp[2:])
            conv[-1] = -(hc * w * h / 6.0) * (2.0 * Tp[-1] + Tp[-2])
        else:
            conv = -hc * w * h * Tp
            conv[-1] = -hc * w * h / 2.0 * Tp[-1]
        m = np.full(nx + 1, m_in)
        m[-1] = m_in / 2.0
        Tn = T + dt * (cond + conv) / m
        Tn[0] = Ts
        T = Tn
    return T
