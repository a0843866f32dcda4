"""FP64 CPU oracle of the fluid flow in the fractures and of the coupled
hydro-mechanical Jacobian (Sec. 3.2: weak form eq. weak_form_flow, the discrete system
eq. flow_discretized with its element matrices V, S, L and f_f, the residual eq.
res_flow; Sec. 3.3: the coupled residuals r_m, r_f and the 2x2 block Jacobian of
Sec. 3.3.1 with A11 = E - eta/dt - C^ep, A12 = N_p, A21, A22; the upper block
triangular preconditioner P_up and its approximate Schur complement with
A11~ = diag(A11)).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path; it shares no
code with the CUDA library.

Readings taken where the paper is silent or fixes another element type:
  F1 pressure: linear shape functions on triangles (the paper's P1 elements) and
     bilinear ones on rectangles, nodes at the vertices, one node per distinct vertex
     position, so elements share a node where their vertices coincide (also across
     intersecting planes and between the two shapes);
  F2 permeability: the cubic law, w k(w) / mu_f = w^3 / (12 mu_f) with w = w_o + delta_n,
     constant over an element (the DD is piecewise constant); 1/M constant;
  F3 the Jacobian is the exact derivative of the discrete residuals: A21 also carries
     the derivative of dt L(delta) (p^n - p^o), which the residual eq. res_flow contains;
  F4 the pore pressure at a collocation point is the interpolation at the element's
     centroid, the mean of its nodal pressures: N_p holds 1/4 (rectangle) or 1/3
     (triangle) on the element's normal row;
  F5 no flux through the outer boundary (the natural condition of the weak form); f_f
     given as nodal volume rates.
Element integrals by quadrature exact for these integrands: 2 x 2 Gauss-Legendre on a
rectangle; on a triangle the three edge-midpoint rule (exact for quadratics), with the
linear shape functions from the vertices' Vandermonde system.
Dense matrices: for the small cases of the tests.
"""
from __future__ import annotations

import numpy as np

# local node order: (-a, -b), (+a, -b), (+a, +b), (-a, +b) in the element's (s1, s2) frame
XI = np.array([-1.0, 1.0, 1.0, -1.0])
ETA = np.array([-1.0, -1.0, 1.0, 1.0])
GAUSS = np.array([-1.0, 1.0]) / np.sqrt(3.0)


def shape(xi, eta):
    """Bilinear shape functions N_i and their derivatives in (xi, eta)."""
    N = 0.25 * (1 + XI * xi) * (1 + ETA * eta)
    dxi = 0.25 * XI * (1 + ETA * eta)
    deta = 0.25 * ETA * (1 + XI * xi)
    return N, dxi, deta


def element_matrices(a, b):
    """On a rectangle of half sides a, b: mass m_ij = int N_i N_j dS, stiffness
    k_ij = int grad N_i . grad N_j dS and load v_i = int N_i dS."""
    m = np.zeros((4, 4))
    k = np.zeros((4, 4))
    v = np.zeros(4)
    J = a * b  # dS = a b dxi deta
    for xi in GAUSS:
        for eta in GAUSS:
            N, dxi, deta = shape(xi, eta)
            gx, gy = dxi / a, deta / b
            m += np.outer(N, N) * J
            k += (np.outer(gx, gx) + np.outer(gy, gy)) * J
            v += N * J
    return m, k, v


def tri_element_matrices(V):
    """On the triangle with vertices V (3 x 3, global, in the element's node order):
    mass, stiffness and load by the edge-midpoint rule; N_i = c0 + c1 x + c2 y in an
    orthonormal frame of the triangle's plane."""
    V = np.asarray(V, dtype=float)
    e1 = V[1] - V[0]
    n = np.cross(e1, V[2] - V[0])
    area = 0.5 * np.linalg.norm(n)
    t1 = e1 / np.linalg.norm(e1)
    t2 = np.cross(n / np.linalg.norm(n), t1)
    xy = np.stack([(V - V[0]) @ t1, (V - V[0]) @ t2], axis=1)
    C = np.linalg.inv(np.column_stack([np.ones(3), xy]))  # column i: coefficients of N_i
    grad = C[1:, :].T                                      # (3 nodes, 2)
    pts = 0.5 * (xy + np.roll(xy, -1, axis=0))            # edge midpoints
    N = np.column_stack([np.ones(3), pts]) @ C             # (3 points, 3 nodes)
    m = (area / 3.0) * N.T @ N
    k = area * grad @ grad.T
    v = (area / 3.0) * N.sum(axis=0)
    return m, k, v


def element_set(conn, a, b, shape=None, tri=None):
    """Per element: its nodes and its (mass, stiffness, load) matrices -- bilinear on a
    rectangle (conn row of 4), linear on a triangle (the first 3 of its conn row)."""
    out = []
    for e in range(conn.shape[0]):
        if shape is not None and shape[e] == 1:
            m, k, v = tri_element_matrices(np.asarray(tri[e]).reshape(3, 3))
            out.append((np.asarray(conn[e][:3]), m, k, v))
        else:
            m, k, v = element_matrices(a[e], b[e])
            out.append((np.asarray(conn[e][:4]), m, k, v))
    return out


def conductance(w, mu):
    """w k(w) / mu_f with the cubic law k = w^2 / 12 (reading F2), and its derivative."""
    return w ** 3 / (12.0 * mu), 3.0 * w ** 2 / (12.0 * mu)


def assemble(conn, n_nodes, a, b, dn, M, mu, w0, shape=None, tri=None):
    """Global V (n_nodes x N: per element's normal DD), S = sum (w/M) m^e and
    L = sum (w^3 / 12 mu) k^e at the openings w = w0 + dn (eq. flow_discretized)."""
    N = conn.shape[0]
    V = np.zeros((n_nodes, N))
    S = np.zeros((n_nodes, n_nodes))
    L = np.zeros((n_nodes, n_nodes))
    for e, (idx, m, k, v) in enumerate(element_set(conn, a, b, shape, tri)):
        w = w0 + dn[e]
        c, _ = conductance(w, mu)
        V[idx, e] += v
        S[np.ix_(idx, idx)] += (w / M) * m
        L[np.ix_(idx, idx)] += c * k
    return V, S, L


def flow_residual(conn, n_nodes, a, b, dn_old, ddn, dp, pn, f, M, mu, w0, dt, shape=None, tri=None):
    """r_f = V ddn + (S + dt L) dp + dt L pn - dt f (eq. res_flow) with S and L at the
    openings of t^(n+1), w = w0 + dn_old + ddn; pn = p^n - p^o."""
    V, S, L = assemble(conn, n_nodes, a, b, dn_old + ddn, M, mu, w0, shape, tri)
    return V @ ddn + (S + dt * L) @ dp + dt * L @ pn - dt * f


def jacobian_blocks(conn, n_nodes, a, b, dn, dp, pn, M, mu, w0, dt, shape=None, tri=None):
    """A12 = N_p (3N x n_nodes), A21 = d r_f / d Delta delta (n_nodes x 3N), A22 =
    S + dt L (n_nodes x n_nodes) at the openings w = w0 + dn (Sec. 3.3.1, readings F3,
    F4).  Only the normal DD of an element enters r_f."""
    N = conn.shape[0]
    A12 = np.zeros((3 * N, n_nodes))
    A21 = np.zeros((n_nodes, 3 * N))
    V, S, L = assemble(conn, n_nodes, a, b, dn, M, mu, w0, shape, tri)
    for e, (idx, m, k, v) in enumerate(element_set(conn, a, b, shape, tri)):
        A12[3 * e + 2, idx] += 1.0 / len(idx)
        w = w0 + dn[e]
        _, dc = conductance(w, mu)
        # d/d delta_n of V delta + S dp + dt L (dp + pn) on the element's nodes
        A21[idx, 3 * e + 2] += v + (m @ dp[idx]) / M + dt * dc * (k @ (dp[idx] + pn[idx]))
    return A12, A21, S + dt * L


def coupled(A11, A12, A21, A22):
    """The 2 x 2 block Jacobian [[A11, A12], [A21, A22]]."""
    return np.block([[A11, A12], [A21, A22]])


def schur_diag(A11, A12, A21, A22):
    """S~ = A22 - A21 diag(A11)^-1 A12 (Sec. 3.3.1, the first approximation of A11)."""
    d = np.diag(A11)
    return A22 - A21 @ (A12 / d[:, None])


def apply_pup_inverse(A11, A12, Sd, y, n1):
    """z = P_up^-1 y with exact solves: z2 = S~^-1 y2, z1 = A11^-1 (y1 - A12 z2)."""
    z2 = np.linalg.solve(Sd, y[n1:])
    z1 = np.linalg.solve(A11, y[:n1] - A12 @ z2)
    return np.concatenate([z1, z2])
