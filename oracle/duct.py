"""Fully developed MHD flow in a rectangular duct with thin conducting walls: the reference solutions
for the duct tests.  TEST INFRASTRUCTURE ONLY.

The paper names flows with side (Shercliff) layers -- ducts whose walls run parallel to the applied
field -- as the next case for its closures (end of Sec. VII, Sec. IX).  Here the duct axis is x
(periodic), the Hartmann walls are the planes y = -a, +a (normal to the applied field B0 along y) and
the side walls the planes z = -b, +b.  Fully developed, u = u_x(y, z) and the induced field is
B_x(y, z), and with rho = mu_m = 1, sigma = 1/eta the steady equations are

    nu (u_yy + u_zz) + B0 dB_x/dy + F = 0,     eta (B_yy + B_zz) + B0 du/dy = 0,

(the x components of the momentum balance with the Lorentz force J x B = B0 dB_x/dy and of the
induction equation), with u = 0 on every wall and on each wall the Shercliff thin-wall condition of
Eq. ShercliffBClocalcoordinate for the tangential induced field,  B_x + c a dB_x/dn = 0,  dn along the
outward normal, c the wall's conductance ratio.  Every wall's ratio is taken relative to the same
length a (the Hartmann half-width), so c a = sigma_w t_w / sigma for each wall; c = inf is the
perfectly conducting limit dB_x/dn = 0.

Two independent ways to the solution:
  hunt_series  -- insulating side walls (c_side = 0) and equal Hartmann walls of ratio c: then u and
                  B_x both vanish at z = +-b, cos((2k+1) pi z/(2b)) is a common eigenbasis and each
                  mode is a pair of constant-coefficient ODEs in y, solved in closed form below (the
                  structure of Hunt's classical duct solution, derived here from the equations).
  fd_solve     -- any four walls: second-order finite differences on a node grid, ghost nodes for the
                  Robin conditions, one sparse linear solve.
"""
import math

import numpy as np


def _ch(m, y, a):
    """cosh(m y)/cosh(m a) without overflow (|y| <= a)."""
    m = np.abs(m)
    ay = np.abs(y)
    return np.exp(m * (ay - a)) * (1.0 + np.exp(-2.0 * m * ay)) / (1.0 + np.exp(-2.0 * m * a))


def _sh(m, y, a):
    """sinh(m y)/cosh(m a) without overflow (|y| <= a)."""
    s = np.sign(m) * np.sign(y)
    m = np.abs(m)
    ay = np.abs(y)
    return s * np.exp(m * (ay - a)) * (1.0 - np.exp(-2.0 * m * ay)) / (1.0 + np.exp(-2.0 * m * a))


def _th(m, a):
    return math.tanh(m * a)


def hunt_series(y, z, a, b, B0, nu, eta, F, c, nterms=4000):
    """u_x(y, z), B_x(y, z) for insulating side walls and Hartmann walls of ratio c (both).

    Mode k: u = U_k(y) cos(l z), B = B_k(y) cos(l z), l = (2k+1) pi/(2b), and the body force's
    coefficient F_k = 4 F (-1)^k/((2k+1) pi).  The modal equations
        nu (U'' - l^2 U) + B0 B' + F_k = 0,   eta (B'' - l^2 B) + B0 U' = 0
    have the particular solution U = F_k/(nu l^2), B = 0, and exponential solutions e^{m y} with
    (m^2 - l^2)^2 = H^2 m^2, H = B0/sqrt(nu eta) = Ha/a: m^2 - l^2 = +H m (roots m1 = H/2 + s,
    m2 = H/2 - s, s = sqrt(H^2/4 + l^2), with B = -kappa U) or -H m (roots -m1, -m2, B = +kappa U),
    kappa = sqrt(nu/eta).  The even-u, odd-B combination is
        U = F_k/(nu l^2) + P cosh(m1 y)/cosh(m1 a) + Q cosh(m2 y)/cosh(m2 a),
        B = -kappa [P sinh(m1 y)/cosh(m1 a) + Q sinh(m2 y)/cosh(m2 a)],
    and U(a) = 0, B(a) + c a B'(a) = 0 (the condition at -a then holds by symmetry) give
        P + Q = -F_k/(nu l^2),   P (tanh(m1 a) + c a m1) + Q (tanh(m2 a) + c a m2) = 0
    (for c = inf the second row divided by c: P m1 + Q m2 = 0)."""
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    H = B0 / math.sqrt(nu * eta)
    kappa = math.sqrt(nu / eta)
    u = np.zeros(np.broadcast(y, z).shape)
    bx = np.zeros_like(u)
    for k in range(nterms):
        lam = (2 * k + 1) * math.pi / (2.0 * b)
        Fk = 4.0 * F * (-1) ** k / ((2 * k + 1) * math.pi)
        Up = Fk / (nu * lam * lam)
        s = math.sqrt(0.25 * H * H + lam * lam)
        m1, m2 = 0.5 * H + s, 0.5 * H - s
        if math.isinf(c):
            r1, r2 = m1, m2
        else:
            r1, r2 = _th(m1, a) + c * a * m1, _th(m2, a) + c * a * m2
        det = r2 - r1
        P = -Up * r2 / det
        Q = Up * r1 / det
        cz = np.cos(lam * z)
        u = u + cz * (Up + P * _ch(m1, y, a) + Q * _ch(m2, y, a))
        bx = bx - kappa * cz * (P * _sh(m1, y, a) + Q * _sh(m2, y, a))
    return u, bx


def fd_solve(a, b, B0, nu, eta, F, c_bot, c_top, c_back, c_front, ny, nz, field_axis="y"):
    """Second-order finite-difference solution on the node grid y_i = -a + i h_y (i = 0..ny),
    z_j = -b + j h_z (j = 0..nz).  Returns (y, z, u[ny+1, nz+1], B[ny+1, nz+1]).

    c_bot, c_top: ratios of the walls y = -a, +a; c_back, c_front: of z = -b, +b.  field_axis: the
    direction of the applied field ("y": the duct of this module; "z": the same problem turned by a
    right angle, B0 along z, whose derivative terms are B0 dB/dz and B0 du/dz -- used to check the
    z-wall code against the series).  u is 0 on the boundary nodes; the momentum equation holds at the
    interior nodes with centred differences.  The induction equation holds at every node where B is
    not fixed: at a wall node the second difference across the wall uses a ghost node from the centred
    Robin condition B + c a dB/dn = 0 (ghost = inner neighbour - 2 h B/(c a) along the outward
    normal; c = inf: ghost = inner neighbour), and at a wall of c = 0 the node value is B = 0.  The
    field-direction derivative of u at a wall normal to the field is the one-sided second-order
    difference (u = 0 on the wall); along walls parallel to the field u = 0, so it vanishes there."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.linalg import spsolve

    hy, hz = 2.0 * a / ny, 2.0 * b / nz
    NY, NZ = ny + 1, nz + 1
    iu = -np.ones((NY, NZ), dtype=np.int64)
    cnt = 0
    for i in range(1, ny):
        for j in range(1, nz):
            iu[i, j] = cnt
            cnt += 1
    nu_unk = cnt
    ib = np.arange(NY * NZ, dtype=np.int64).reshape(NY, NZ) + nu_unk
    nunk = nu_unk + NY * NZ
    rows, cols, vals = [], [], []
    rhs = np.zeros(nunk)
    along_y = field_axis == "y"
    hf = hy if along_y else hz

    def add(r, c_, v):
        rows.append(r)
        cols.append(c_)
        vals.append(v)

    def nb(i, j, d):
        """Neighbour (i, j) + d steps along the field axis."""
        return (i + d, j) if along_y else (i, j + d)

    # momentum at interior nodes
    for i in range(1, ny):
        for j in range(1, nz):
            r = iu[i, j]
            add(r, r, nu * (-2.0 / hy ** 2 - 2.0 / hz ** 2))
            for (ii, jj, w) in ((i - 1, j, nu / hy ** 2), (i + 1, j, nu / hy ** 2),
                                (i, j - 1, nu / hz ** 2), (i, j + 1, nu / hz ** 2)):
                if iu[ii, jj] >= 0:
                    add(r, iu[ii, jj], w)
            add(r, ib[nb(i, j, 1)], B0 / (2.0 * hf))
            add(r, ib[nb(i, j, -1)], -B0 / (2.0 * hf))
            rhs[r] = -F

    def robin_weight(c, h):
        """Second difference across a wall node: (2 B_in - 2 B - 2 h B/(c a))/h^2."""
        return 0.0 if math.isinf(c) else 2.0 * h / (c * a)

    for i in range(NY):
        for j in range(NZ):
            r = ib[i, j]
            # a node on a wall of c = 0 holds B = 0
            fixed = ((i == 0 and c_bot == 0.0) or (i == ny and c_top == 0.0) or
                     (j == 0 and c_back == 0.0) or (j == nz and c_front == 0.0))
            if fixed:
                add(r, r, 1.0)
                continue
            diag = 0.0
            # y direction
            if i == 0:
                add(r, ib[1, j], eta * 2.0 / hy ** 2)
                diag += eta * (-2.0 - robin_weight(c_bot, hy)) / hy ** 2
            elif i == ny:
                add(r, ib[ny - 1, j], eta * 2.0 / hy ** 2)
                diag += eta * (-2.0 - robin_weight(c_top, hy)) / hy ** 2
            else:
                add(r, ib[i - 1, j], eta / hy ** 2)
                add(r, ib[i + 1, j], eta / hy ** 2)
                diag += -2.0 * eta / hy ** 2
            # z direction
            if j == 0:
                add(r, ib[i, 1], eta * 2.0 / hz ** 2)
                diag += eta * (-2.0 - robin_weight(c_back, hz)) / hz ** 2
            elif j == nz:
                add(r, ib[i, nz - 1], eta * 2.0 / hz ** 2)
                diag += eta * (-2.0 - robin_weight(c_front, hz)) / hz ** 2
            else:
                add(r, ib[i, j - 1], eta / hz ** 2)
                add(r, ib[i, j + 1], eta / hz ** 2)
                diag += -2.0 * eta / hz ** 2
            add(r, r, diag)
            # B0 du/d(field axis): zero on the walls parallel to the field (u = 0 along them)
            p, q, last = (i, j, ny) if along_y else (j, i, nz)
            if not (0 < q < (nz if along_y else ny)):
                continue
            if p == 0:
                add(r, iu[nb(i, j, 1)], B0 * 4.0 / (2.0 * hf))
                if iu[nb(i, j, 2)] >= 0:
                    add(r, iu[nb(i, j, 2)], -B0 / (2.0 * hf))
            elif p == last:
                add(r, iu[nb(i, j, -1)], -B0 * 4.0 / (2.0 * hf))
                if iu[nb(i, j, -2)] >= 0:
                    add(r, iu[nb(i, j, -2)], B0 / (2.0 * hf))
            else:
                if iu[nb(i, j, 1)] >= 0:
                    add(r, iu[nb(i, j, 1)], B0 / (2.0 * hf))
                if iu[nb(i, j, -1)] >= 0:
                    add(r, iu[nb(i, j, -1)], -B0 / (2.0 * hf))
    A = coo_matrix((vals, (rows, cols)), shape=(nunk, nunk)).tocsr()
    sol = spsolve(A, rhs)
    u = np.zeros((NY, NZ))
    u[1:ny, 1:nz] = sol[:nu_unk].reshape(ny - 1, nz - 1)
    B = sol[nu_unk:].reshape(NY, NZ)
    y = -a + hy * np.arange(NY)
    z = -b + hz * np.arange(NZ)
    return y, z, u, B


def fd_on_lattice(ny_lat, nz_lat, B0, nu, eta, F, c_bot, c_top, c_back, c_front, refine=4):
    """fd_solve on a grid whose nodes include the link-based lattice's nodes y_j = -a + j + 1/2,
    z_k = -b + k + 1/2 (a = ny_lat/2, b = nz_lat/2): spacing h = 1/(2 refine), sampled there.
    Returns u, B of shape (ny_lat, nz_lat)."""
    a, b = 0.5 * ny_lat, 0.5 * nz_lat
    m = 2 * refine
    y, z, u, B = fd_solve(a, b, B0, nu, eta, F, c_bot, c_top, c_back, c_front, ny_lat * m, nz_lat * m)
    iy = (2 * np.arange(ny_lat) + 1) * refine
    iz = (2 * np.arange(nz_lat) + 1) * refine
    return u[np.ix_(iy, iz)], B[np.ix_(iy, iz)]


def fd_on_lattice_extrapolated(ny_lat, nz_lat, B0, nu, eta, F, c_bot, c_top, c_back, c_front, refine=1):
    """Richardson extrapolation of fd_on_lattice from spacings h = 1/(2 refine) and h/2:
    (4 fine - coarse)/3 removes the O(h^2) term of the second-order solution."""
    uc, Bc = fd_on_lattice(ny_lat, nz_lat, B0, nu, eta, F, c_bot, c_top, c_back, c_front, refine=refine)
    uf, Bf = fd_on_lattice(ny_lat, nz_lat, B0, nu, eta, F, c_bot, c_top, c_back, c_front, refine=2 * refine)
    return (4.0 * uf - uc) / 3.0, (4.0 * Bf - Bc) / 3.0
