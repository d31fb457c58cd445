"""Hex8 linear elasticity on a structured voxel grid, FP64 (oracle; test infrastructure).

The state equation of Eq. 4 is r(z, u) = K(z) u - f = 0 (§III-D).  The paper does not name
the element; the DOF counts of Table 1 fix trilinear hex8 elements with three
displacement components per node.  K(rho) = sum_e E_e(rho_e) * h * K0 assembled over
elements, where K0 is the stiffness of a unit cube with E = 1 and the modified SIMP
interpolation E_e = Emin + rho_e^p (E0 - Emin) holds per element.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# local node a = ax + 2*ay + 4*az  ->  offsets (ax, ay, az), x fastest
LOCAL_NODES = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def lame(E: float, nu: float):
    """Lame constants of an isotropic solid."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def constitutive(E: float, nu: float) -> np.ndarray:
    """6x6 isotropic elasticity matrix, Voigt order (xx, yy, zz, yz, xz, xy) with
    engineering shear strains."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients_natural(xi: np.ndarray) -> np.ndarray:
    """dN_a/dxi_i (8x3) of the trilinear shape functions N_a = prod_i (1 + s_ai xi_i)/8 on
    [-1,1]^3, with s_ai = 2*a_i - 1."""
    s = 2.0 * LOCAL_NODES - 1.0
    G = np.empty((8, 3))
    for a in range(8):
        for i in range(3):
            g = s[a, i] / 8.0
            for j in range(3):
                if j != i:
                    g *= 1.0 + s[a, j] * xi[j]
            G[a, i] = g
    return G


def strain_displacement(dNdx: np.ndarray) -> np.ndarray:
    """6x24 B matrix (element DOF order 3a + c) for physical gradients dNdx (8x3)."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = dNdx[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1] = gz
        B[3, 3 * a + 2] = gy
        B[4, 3 * a + 0] = gz
        B[4, 3 * a + 2] = gx
        B[5, 3 * a + 0] = gy
        B[5, 3 * a + 1] = gx
    return B


def unit_element_stiffness(nu: float) -> np.ndarray:
    """K0 (24x24): stiffness of the unit cube [0,1]^3 with E = 1, 2x2x2 Gauss quadrature
    (exact: the integrand is at most quadratic per axis).  Element of edge h and modulus
    E has stiffness h * E * K0."""
    D = constitutive(1.0, nu)
    g = 1.0 / np.sqrt(3.0)
    K0 = np.zeros((24, 24))
    for gz in (-g, g):
        for gy in (-g, g):
            for gx in (-g, g):
                dNdxi = shape_gradients_natural(np.array([gx, gy, gz]))
                dNdx = 2.0 * dNdxi            # x = (xi + 1)/2 on the unit cube
                B = strain_displacement(dNdx)
                K0 += B.T @ D @ B * (1.0 / 8.0)  # det J = 1/8, Gauss weights 1
    return 0.5 * (K0 + K0.T)


def element_dofs(nx: int, ny: int, nz: int) -> np.ndarray:
    """Global DOF indices int64[N_el, 24] in element order 3a + c, SoA global numbering
    c*N_n + n with n = i + (nx+1)*(j + (ny+1)*k)."""
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    edof = np.empty((nx * ny * nz, 24), dtype=np.int64)
    for a in range(8):
        ax, ay, az = LOCAL_NODES[a]
        node = (i + ax) + (nx + 1) * ((j + ay) + (ny + 1) * (k + az))
        for c in range(3):
            edof[:, 3 * a + c] = c * nn + node
    return edof


def simp_modulus(rho: np.ndarray, E0: float, Emin: float, penal: float) -> np.ndarray:
    """Modified SIMP interpolation E = Emin + rho^p (E0 - Emin)."""
    return Emin + np.power(rho, penal) * (E0 - Emin)


def assemble(nx: int, ny: int, nz: int, Ee: np.ndarray, h: float, K0: np.ndarray) -> sp.csr_matrix:
    """Sparse K = sum_e h E_e K0 (all DOFs, no boundary conditions), CSR, FP64."""
    edof = element_dofs(nx, ny, nz)
    ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    rows = np.repeat(edof, 24, axis=1).ravel()
    cols = np.tile(edof, (1, 24)).ravel()
    vals = ((h * np.asarray(Ee, dtype=np.float64))[:, None, None] * K0[None, :, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    return K


def apply_elementwise(nx: int, ny: int, nz: int, Ee: np.ndarray, h: float, K0: np.ndarray,
                      x: np.ndarray, edof: np.ndarray | None = None) -> np.ndarray:
    """y = K x computed element by element: gather x_e, multiply by h E_e K0, add back.
    Same operator as ``assemble`` without forming the matrix (used on large grids)."""
    if edof is None:
        edof = element_dofs(nx, ny, nz)
    ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    Xe = x[edof]
    Ye = (Xe @ K0) * (h * np.asarray(Ee, dtype=np.float64))[:, None]
    return np.bincount(edof.ravel(), weights=Ye.ravel(), minlength=ndof)


def diagonal_elementwise(nx: int, ny: int, nz: int, Ee: np.ndarray, h: float, K0: np.ndarray,
                         edof: np.ndarray | None = None) -> np.ndarray:
    """diag(K), accumulated element by element."""
    if edof is None:
        edof = element_dofs(nx, ny, nz)
    ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    de = np.diag(K0)[None, :] * (h * np.asarray(Ee, dtype=np.float64))[:, None]
    return np.bincount(edof.ravel(), weights=de.ravel(), minlength=ndof)


def element_bilinear(nx: int, ny: int, nz: int, w: np.ndarray, u: np.ndarray, K0: np.ndarray,
                     edof: np.ndarray | None = None) -> np.ndarray:
    """w_e^T K0 u_e per element (unit modulus, unit size)."""
    if edof is None:
        edof = element_dofs(nx, ny, nz)
    return np.einsum("ei,ij,ej->e", w[edof], K0, u[edof])


def element_energy(nx: int, ny: int, nz: int, u: np.ndarray, K0: np.ndarray,
                   edof: np.ndarray | None = None) -> np.ndarray:
    """u_e^T K0 u_e per element (unit modulus, unit size)."""
    if edof is None:
        edof = element_dofs(nx, ny, nz)
    Ue = u[edof]
    return np.einsum("ei,ij,ej->e", Ue, K0, Ue)
