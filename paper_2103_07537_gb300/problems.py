"""Seeded synthetic coupled block systems: the inputs that both the CUDA path and
the FP64 oracle solve.

This module generates inputs only.  It holds none of the multigrid method's
arithmetic (no aggregation, smoothing, transfer, Galerkin product or Krylov
step); it assembles Q1 finite-element matrices on uniform grids and draws
right-hand sides and coefficients from a counter-based generator.

The paper's own systems come from a stabilised finite-element resistive-MHD
code (Sec. 2, the 4x4 block Jacobian) that is not available, so these Q1
systems stand in for them with the same block structure:

* ``stokes2d``: Q1-Q1 pressure-stabilised Stokes on an N x N cell grid of the
  unit square, dofs per node (u, v, p), one field block.
* ``mhd2d``: the 2x2 split of Sec. 3 (Navier-Stokes {u, v, p} against Maxwell
  {Bx, By, psi}), dofs per node (u, v, p, Bx, By, psi), two field blocks, the
  B-u coupling being a linearised cross product with a frozen smooth field B0.
* ``stokes3d``: Q1-Q1 stabilised Stokes on an N^3 hex grid, dofs (u, v, w, p).
* ``mhd2d_q2q1``: the same two blocks on different element spaces (the
  mixed-element example of Sec. 5): {u, v, p} on biquadratic Q2 nodes,
  {Bx, By, psi} on bilinear Q1 vertices, so the two fields live on disjoint
  node sets (hydrodynamic nodes first), three dofs per node in both.

Block-row layout (shared by every consumer): nodes are numbered row-major
(x fastest); block CSR over nodes with column indices ascending; each stored
block is b x b, row-major; the dofs of a node are interleaved in field order.
The pattern is structural (the full 9- or 27-point node stencil); Dirichlet
rows and columns are replaced by identity rows and columns without removing
stored zeros.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) in counter form: value k of a
stream with seed s is mix(s + (k + 1) * 0x9E3779B97F4A7C15), so any language
reproduces it bit for bit.  A double in [0, 1) is (v >> 11) * 2^-53.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Values start .. start+count-1 of the splitmix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    v = splitmix64(seed, start, count) >> np.uint64(11)
    return v.astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, start: int, count: int) -> np.ndarray:
    return 2.0 * uniform01(seed, start, count) - 1.0


@dataclasses.dataclass
class BlockSystem:
    """A block-CSR system A x = rhs with a field-to-dof map."""

    name: str
    n_nodes: int
    b: int
    row_ptr: np.ndarray  # int32 [n_nodes + 1]
    col_idx: np.ndarray  # int32 [nnzb]
    vals: np.ndarray  # float64 [nnzb, b, b]
    rhs: np.ndarray  # float64 [n_nodes * b]
    field_of_dof: list
    params: dict
    # fields on disjoint node sets: field g owns nodes node_field_off[g] ..
    # node_field_off[g+1]-1 with all their dofs (None: co-located fields)
    node_field_off: list | None = None

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_unknowns(self) -> int:
        return self.n_nodes * self.b

    def to_scipy(self):
        """The system matrix as a scipy BSR matrix (test convenience)."""
        import scipy.sparse as sp

        return sp.bsr_matrix(
            (self.vals, self.col_idx, self.row_ptr),
            shape=(self.n_unknowns, self.n_unknowns),
        )

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


# ----------------------------------------------------------------------------
# structured node graphs
# ----------------------------------------------------------------------------

def _stencil_pattern(dims):
    """Block pattern of the full node stencil on a structured grid.

    ``dims`` = nodes per side, x first.  Returns row_ptr, col_idx, and
    ``pos[i, o]`` = index of the stored block (i, neighbour o) or -1, where
    o enumerates offsets in (dz, dy, dx) lexicographic order; that order gives
    ascending column indices.
    """
    d = len(dims)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(d, -1)[::-1]  # coords[0] = x
    offsets = np.array(np.meshgrid(*([[-1, 0, 1]] * d), indexing="ij")).reshape(d, -1)
    offsets = offsets[::-1]  # offsets[0] = dx; enumeration is (dz, dy, dx) lexicographic
    strides = np.cumprod([1] + list(dims[:-1]))
    n_off = offsets.shape[1]
    valid = np.ones((n, n_off), dtype=bool)
    nbr = np.zeros((n, n_off), dtype=np.int64)
    for a in range(d):
        c = coords[a][:, None] + offsets[a][None, :]
        valid &= (c >= 0) & (c < dims[a])
        nbr += c * strides[a]
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    col_idx = nbr[valid].astype(np.int32)
    rank = np.cumsum(valid, axis=1) - 1
    pos = np.where(valid, row_ptr[:-1, None] + rank, -1)
    return row_ptr.astype(np.int32), col_idx, pos, coords, offsets


def _offset_code(delta):
    """Index of an offset vector (dx, dy[, dz]) in the stencil enumeration."""
    code = 0
    for a in reversed(range(len(delta))):
        code = code * 3 + (delta[a] + 1)
    return code


# ----------------------------------------------------------------------------
# Q1 reference element
# ----------------------------------------------------------------------------

def _q1_reference(d):
    """Shape values and reference gradients of the d-linear element at the
    2^d Gauss points (weights 1) of [-1, 1]^d.

    Local node l has bits (lx, ly[, lz]) = l & 1, (l >> 1) & 1, (l >> 2) & 1.
    Returns phi[q, l], dphi[q, l, a] and the reference points xi[q, a].
    """
    g = 1.0 / math.sqrt(3.0)
    nl = 2 ** d
    pts = np.array(np.meshgrid(*([[-g, g]] * d), indexing="ij")).reshape(d, -1).T
    sgn = np.array([[1.0 if (l >> a) & 1 else -1.0 for a in range(d)] for l in range(nl)])
    nq = pts.shape[0]
    phi = np.ones((nq, nl))
    dphi = np.ones((nq, nl, d))
    for a in range(d):
        fac = 1.0 + sgn[None, :, a] * pts[:, a, None]  # [q, l]
        phi *= fac / 2.0
        for c in range(d):
            if c == a:
                dphi[:, :, c] *= sgn[None, :, a] / 2.0
            else:
                dphi[:, :, c] *= fac / 2.0
    return phi, dphi, pts


def _element_nodes(cell_dims):
    """Global node of every (element, local node), row-major numbering."""
    d = len(cell_dims)
    node_dims = [c + 1 for c in cell_dims]
    strides = np.cumprod([1] + node_dims[:-1])
    ecoords = np.indices(cell_dims[::-1]).reshape(d, -1)[::-1]
    nl = 2 ** d
    out = np.zeros((ecoords.shape[1], nl), dtype=np.int64)
    for l in range(nl):
        g = np.zeros(ecoords.shape[1], dtype=np.int64)
        for a in range(d):
            g += (ecoords[a] + ((l >> a) & 1)) * strides[a]
        out[:, l] = g
    return out, ecoords


def _scatter(vals, pos, elem_nodes, d, blocks_of_pair):
    """Add element blocks into the BSR value array.

    ``blocks_of_pair(la, lc)`` returns a [b, b] block (same for every element)
    or a [E, b, b] array.  For a fixed local pair (la, lc) every element hits
    a different stored block, so a plain fancy-index add is exact.
    """
    nl = 2 ** d
    for la in range(nl):
        for lc in range(nl):
            delta = [((lc >> a) & 1) - ((la >> a) & 1) for a in range(d)]
            code = _offset_code(delta)
            idx = pos[elem_nodes[:, la], code]
            vals[idx] += blocks_of_pair(la, lc)


def _apply_dirichlet(vals, row_ptr, col_idx, pos, center_code, constrained):
    """Identity rows and columns for constrained dofs; the pattern is kept."""
    n = constrained.shape[0]
    counts = np.diff(row_ptr)
    blk_row = np.repeat(np.arange(n), counts)
    vals *= (~constrained[blk_row])[:, :, None]
    vals *= (~constrained[col_idx])[:, None, :]
    diag = pos[:, center_code]
    ii, rr = np.nonzero(constrained)
    vals[diag[ii], rr, rr] = 1.0


def _boundary_nodes(dims):
    d = len(dims)
    coords = np.indices(dims[::-1]).reshape(d, -1)[::-1]
    bnd = np.zeros(coords.shape[1], dtype=bool)
    for a in range(d):
        bnd |= (coords[a] == 0) | (coords[a] == dims[a] - 1)
    return bnd


# ----------------------------------------------------------------------------
# systems
# ----------------------------------------------------------------------------

def _stokes(d, N, seed, nu=1.0):
    """Q1-Q1 Stokes with pressure stabilisation tau = h^2 / (12 nu).

    Rows of node i (velocity components a, pressure):
      u-row: nu K (x) I_d   and  G,   G[(i,a), j] = -int d_a phi_i phi_j
      p-row: -G^T           and  tau K
    Dirichlet velocity on the whole boundary; pressure pinned at node 0.
    """
    h = 1.0 / N
    dims = [N + 1] * d
    b = d + 1
    row_ptr, col_idx, pos, _, _ = _stencil_pattern(dims)
    n = int(np.prod(dims))
    vals = np.zeros((col_idx.shape[0], b, b))
    phi, dphi, _ = _q1_reference(d)
    jac = (h / 2.0) ** d
    grad = dphi * (2.0 / h)  # physical gradients [q, l, a]
    K = np.einsum("qla,qma->lm", grad, grad) * jac
    G = -np.einsum("qla,qm->lam", grad, phi) * jac  # G[la, a, lc]
    tau = h * h / (12.0 * nu)

    def block(la, lc):
        blk = np.zeros((b, b))
        for a in range(d):
            blk[a, a] = nu * K[la, lc]
            blk[a, d] = G[la, a, lc]
            blk[d, a] = -G[lc, a, la]
        blk[d, d] = tau * K[la, lc]
        return blk

    elem_nodes, _ = _element_nodes([N] * d)
    _scatter(vals, pos, elem_nodes, d, block)
    cons = np.zeros((n, b), dtype=bool)
    cons[_boundary_nodes(dims), :d] = True
    cons[0, d] = True
    _apply_dirichlet(vals, row_ptr, col_idx, pos, _offset_code([0] * d), cons)
    rhs = uniform_pm1(seed, 0, n * b)
    name = f"stokes{d}d_{N}"
    return BlockSystem(name, n, b, row_ptr, col_idx, vals, rhs, [0] * b,
                       dict(kind=f"stokes{d}d", N=N, seed=seed, nu=nu, tau=tau, h=h))


def stokes2d(N: int = 32, seed: int = 1, nu: float = 1.0) -> BlockSystem:
    return _stokes(2, N, seed, nu)


def stokes3d(N: int = 64, seed: int = 1, nu: float = 1.0) -> BlockSystem:
    return _stokes(3, N, seed, nu)


N_FOURIER = 4


def frozen_field_coeffs(seed: int, start: int) -> np.ndarray:
    """Stream-function coefficients c[k-1, l-1], k, l = 1..4, uniform[-1, 1]
    damped by 1 / (k^2 + l^2)."""
    c = uniform_pm1(seed, start, N_FOURIER * N_FOURIER).reshape(N_FOURIER, N_FOURIER)
    k = np.arange(1, N_FOURIER + 1)
    return c / (k[:, None] ** 2 + k[None, :] ** 2)


def frozen_field(c: np.ndarray, x: np.ndarray, y: np.ndarray):
    """B0 = curl a, a = sum_kl c_kl sin(k pi x) sin(l pi y) (divergence free)."""
    bx = np.zeros_like(x)
    by = np.zeros_like(x)
    for k in range(1, N_FOURIER + 1):
        for l in range(1, N_FOURIER + 1):
            ckl = c[k - 1, l - 1]
            bx += ckl * l * math.pi * np.sin(k * math.pi * x) * np.cos(l * math.pi * y)
            by -= ckl * k * math.pi * np.cos(k * math.pi * x) * np.sin(l * math.pi * y)
    return bx, by


def mhd2d(N: int = 128, seed: int = 1, nu: float | None = None, eta: float | None = None,
          eta_range=(1e-3, 1.0), nu_range=(1e-3, 1.0), eta_cells: bool = False) -> BlockSystem:
    """Two-field 2D system with the block structure of the paper's 4x4 MHD
    Jacobian (Sec. 2) grouped into the 2x2 split of Sec. 3.

    Dofs per node: (u, v, p | Bx, By, psi); field map [0, 0, 0, 1, 1, 1].
      u-row:  nu K (x) I_2,  G,        Z,              0
      p-row:  -G^T,          tau_p K,  0,              0
      B-row:  Y,             0,        eta K (x) I_2,  G
      psi-row: 0,            0,        -G^T,           tau_psi K
    with Y[(i,a),(j,c)] = int curl(phi_i e_a) . (phi_j e_c x B0)_z, Z = -Y^T,
    tau_p = h^2 / (12 nu), tau_psi = h^2 / (12 eta).  nu and eta are drawn
    log-uniformly unless given.  Dirichlet u, B and psi on the boundary;
    pressure pinned at node 0.

    Stream layout for ``seed``: [0] nu, [1] eta, [2..17] Fourier
    coefficients of B0, then the right-hand side (uniform[-1, 1]); with
    ``eta_cells`` the resistivity of every cell is drawn log-uniformly from
    ``eta_range`` from the N*N values that follow the right-hand side (cells
    x-fastest), and tau_psi follows it cell by cell.
    """
    d = 2
    h = 1.0 / N
    dims = [N + 1] * d
    b = 6
    u01 = uniform01(seed, 0, 2)
    lo, hi = math.log10(nu_range[0]), math.log10(nu_range[1])
    if nu is None:
        nu = 10.0 ** (lo + (hi - lo) * u01[0])
    lo, hi = math.log10(eta_range[0]), math.log10(eta_range[1])
    if eta is None:
        eta = 10.0 ** (lo + (hi - lo) * u01[1])
    coef = frozen_field_coeffs(seed, 2)
    rhs_start = 2 + N_FOURIER * N_FOURIER

    row_ptr, col_idx, pos, _, _ = _stencil_pattern(dims)
    n = int(np.prod(dims))
    vals = np.zeros((col_idx.shape[0], b, b))
    phi, dphi, pts = _q1_reference(d)
    jac = (h / 2.0) ** d
    grad = dphi * (2.0 / h)
    K = np.einsum("qla,qma->lm", grad, grad) * jac
    G = -np.einsum("qla,qm->lam", grad, phi) * jac
    if eta_cells:
        u = uniform01(seed, rhs_start + (N + 1) ** d * b, N ** d)
        eta = 10.0 ** (lo + (hi - lo) * u)  # [E], one per cell (x fastest)
    tau_p = h * h / (12.0 * nu)
    tau_s = h * h / (12.0 * eta)

    elem_nodes, ecoords = _element_nodes([N] * d)
    # B0 at the quadrature points of every element, scaled to max |B0| = 1
    xq = (ecoords[0][:, None] + (pts[None, :, 0] + 1.0) / 2.0) * h
    yq = (ecoords[1][:, None] + (pts[None, :, 1] + 1.0) / 2.0) * h
    bx, by = frozen_field(coef, xq, yq)
    scale = np.sqrt(bx * bx + by * by).max()
    bx /= scale
    by /= scale
    # curl(phi e_x) = -d_y phi, curl(phi e_y) = d_x phi
    curl = np.stack([-grad[:, :, 1], grad[:, :, 0]], axis=-1)  # [q, l, a]
    # (phi e_x x B0)_z = phi By, (phi e_y x B0)_z = -phi Bx
    cross = np.stack([phi[None] * by[:, :, None], -phi[None] * bx[:, :, None]], axis=-1)  # [E, q, l, c]
    Y = np.einsum("qla,eqmc->elamc", curl, cross) * jac  # Y[e, la, a, lc, c]

    def block(la, lc):
        blk = np.zeros((Y.shape[0], b, b))
        for a in range(2):
            blk[:, a, a] = nu * K[la, lc]
            blk[:, a, 2] = G[la, a, lc]
            blk[:, 2, a] = -G[lc, a, la]
            blk[:, 3 + a, 3 + a] = eta * K[la, lc]
            blk[:, 3 + a, 5] = G[la, a, lc]
            blk[:, 5, 3 + a] = -G[lc, a, la]
            for c in range(2):
                blk[:, 3 + a, c] = Y[:, la, a, lc, c]
                blk[:, a, 3 + c] = -Y[:, lc, c, la, a]
        blk[:, 2, 2] = tau_p * K[la, lc]
        blk[:, 5, 5] = tau_s * K[la, lc]
        return blk

    _scatter(vals, pos, elem_nodes, d, block)
    cons = np.zeros((n, b), dtype=bool)
    bnd = _boundary_nodes(dims)
    cons[bnd, 0:2] = True
    cons[bnd, 3:6] = True
    cons[0, 2] = True
    _apply_dirichlet(vals, row_ptr, col_idx, pos, _offset_code([0] * d), cons)
    rhs = uniform_pm1(seed, rhs_start, n * b)
    return BlockSystem(f"mhd2d_{N}_s{seed}", n, b, row_ptr, col_idx, vals, rhs,
                       [0, 0, 0, 1, 1, 1],
                       dict(kind="mhd2d", N=N, seed=seed, nu=nu, eta="per-cell" if eta_cells else eta,
                            tau_p=tau_p, tau_psi="per-cell" if eta_cells else tau_s, h=h))


def _lagrange_1d(order, xi):
    """Values and derivatives of the 1D Lagrange basis of ``order`` (1 or 2)
    on the equispaced nodes of [-1, 1], at the points ``xi``."""
    if order == 1:
        v = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0], axis=-1)
        d = np.stack([np.full_like(xi, -0.5), np.full_like(xi, 0.5)], axis=-1)
    else:
        v = np.stack([xi * (xi - 1.0) / 2.0, 1.0 - xi * xi, xi * (xi + 1.0) / 2.0], axis=-1)
        d = np.stack([xi - 0.5, -2.0 * xi, xi + 0.5], axis=-1)
    return v, d


def _tensor_basis_2d(order, xi, eta):
    """phi[q, l] and reference gradients dphi[q, l, a] of the tensor-product
    Lagrange element (local node l = lx + (order + 1) * ly) at points (xi, eta)."""
    vx, dx = _lagrange_1d(order, xi)
    vy, dy = _lagrange_1d(order, eta)
    m = order + 1
    phi = np.einsum("qx,qy->qyx", vx, vy).reshape(-1, m * m)
    gx = np.einsum("qx,qy->qyx", dx, vy).reshape(-1, m * m)
    gy = np.einsum("qx,qy->qyx", vx, dy).reshape(-1, m * m)
    return phi, np.stack([gx, gy], axis=-1)


def mhd2d_q2q1(N: int = 64, seed: int = 1, nu: float | None = None, eta: float | None = None,
               eta_range=(1e-3, 1.0), nu_range=(1e-3, 1.0)) -> BlockSystem:
    """The two-field system of ``mhd2d`` on mixed elements: Q2/Q2 for the
    hydrodynamic block {u, v, p} and Q1/Q1 for the magnetic block
    {Bx, By, psi} (the mixed-element example of Sec. 5, in 2D), N x N cells
    of the unit square.

    Nodes: the (2N+1)^2 Q2 nodes first (row-major, x fastest), then the
    (N+1)^2 Q1 vertices; every node carries three dofs of its own field, so
    ``field_of_dof`` is [0, 0, 0] and ``node_field_off`` = [0, n_q2, n_q2 + n_q1].
    Blocks (3 x 3) between
      two Q2 nodes:  [nu K2 (x) I_2, G2; -G2^T, tau_p K2],
      two Q1 nodes:  [eta K1 (x) I_2, G1; -G1^T, tau_psi K1],
      a Q1 row and a Q2 column: Y (B-row against u-column, 2 x 2 corner),
      a Q2 row and a Q1 column: Z = -Y^T,
    with K, G and Y defined as in ``mhd2d`` (Y with Q1 test and Q2 trial
    functions), 3 x 3 Gauss quadrature (exact for these products),
    tau_p = (h/2)^2 / (12 nu) (the Q2 node spacing) and tau_psi = h^2 / (12 eta).
    Dirichlet u and v on the boundary Q2 nodes, B and psi on the boundary Q1
    nodes, pressure pinned at Q2 node 0.  The pattern holds every pair of
    nodes that share a cell.

    Stream layout for ``seed``: [0] nu, [1] eta, [2..17] Fourier coefficients
    of B0, then the right-hand side (uniform[-1, 1]).
    """
    h = 1.0 / N
    b = 3
    m2, m1 = 2 * N + 1, N + 1
    n2, n1 = m2 * m2, m1 * m1
    n = n2 + n1
    u01 = uniform01(seed, 0, 2)
    if nu is None:
        lo, hi = math.log10(nu_range[0]), math.log10(nu_range[1])
        nu = 10.0 ** (lo + (hi - lo) * u01[0])
    if eta is None:
        lo, hi = math.log10(eta_range[0]), math.log10(eta_range[1])
        eta = 10.0 ** (lo + (hi - lo) * u01[1])
    coef = frozen_field_coeffs(seed, 2)
    rhs_start = 2 + N_FOURIER * N_FOURIER

    # 3 x 3 Gauss points of [-1, 1]^2 (x fastest) and their weights
    g = math.sqrt(3.0 / 5.0)
    x1 = np.array([-g, 0.0, g])
    w1 = np.array([5.0, 8.0, 5.0]) / 9.0
    xi = np.tile(x1, 3)
    et = np.repeat(x1, 3)
    wq = np.tile(w1, 3) * np.repeat(w1, 3)
    phi2, dphi2 = _tensor_basis_2d(2, xi, et)
    phi1, dphi1 = _tensor_basis_2d(1, xi, et)
    jac = (h / 2.0) ** 2
    grad2 = dphi2 * (2.0 / h)
    grad1 = dphi1 * (2.0 / h)
    K2 = np.einsum("q,qla,qma->lm", wq, grad2, grad2) * jac
    G2 = -np.einsum("q,qla,qm->lam", wq, grad2, phi2) * jac
    K1 = np.einsum("q,qla,qma->lm", wq, grad1, grad1) * jac
    G1 = -np.einsum("q,qla,qm->lam", wq, grad1, phi1) * jac
    tau_p = (h / 2.0) ** 2 / (12.0 * nu)
    tau_s = h * h / (12.0 * eta)

    # cells, x fastest; their Q2 nodes (lx + 3 ly) and Q1 vertices (lx + 2 ly)
    ex = np.tile(np.arange(N), N)
    ey = np.repeat(np.arange(N), N)
    E = N * N
    q2 = np.zeros((E, 9), dtype=np.int64)
    for ly in range(3):
        for lx in range(3):
            q2[:, lx + 3 * ly] = (2 * ex + lx) + m2 * (2 * ey + ly)
    q1 = np.zeros((E, 4), dtype=np.int64)
    for ly in range(2):
        for lx in range(2):
            q1[:, lx + 2 * ly] = n2 + (ex + lx) + m1 * (ey + ly)

    # B0 at the quadrature points of every cell, scaled to max |B0| = 1
    xq = (ex[:, None] + (xi[None, :] + 1.0) / 2.0) * h
    yq = (ey[:, None] + (et[None, :] + 1.0) / 2.0) * h
    bx, by = frozen_field(coef, xq, yq)
    scale = np.sqrt(bx * bx + by * by).max()
    bx /= scale
    by /= scale
    curl1 = np.stack([-grad1[:, :, 1], grad1[:, :, 0]], axis=-1)  # [q, l1, a]
    cross2 = np.stack([phi2[None] * by[:, :, None], -phi2[None] * bx[:, :, None]], axis=-1)  # [E, q, l2, c]
    Y = np.einsum("q,qla,eqmc->elamc", wq, curl1, cross2) * jac  # [E, l1, a, l2, c]

    # every (row, column, block) contribution, grouped by node pair
    rows, cols, blks = [], [], []
    for la in range(9):
        for lc in range(9):
            blk = np.zeros((b, b))
            for a in range(2):
                blk[a, a] = nu * K2[la, lc]
                blk[a, 2] = G2[la, a, lc]
                blk[2, a] = -G2[lc, a, la]
            blk[2, 2] = tau_p * K2[la, lc]
            rows.append(q2[:, la]); cols.append(q2[:, lc]); blks.append(np.broadcast_to(blk, (E, b, b)))
    for la in range(4):
        for lc in range(4):
            blk = np.zeros((b, b))
            for a in range(2):
                blk[a, a] = eta * K1[la, lc]
                blk[a, 2] = G1[la, a, lc]
                blk[2, a] = -G1[lc, a, la]
            blk[2, 2] = tau_s * K1[la, lc]
            rows.append(q1[:, la]); cols.append(q1[:, lc]); blks.append(np.broadcast_to(blk, (E, b, b)))
    for l1 in range(4):
        for l2 in range(9):
            yb = np.zeros((E, b, b))
            yb[:, :2, :2] = Y[:, l1, :, l2, :]
            rows.append(q1[:, l1]); cols.append(q2[:, l2]); blks.append(yb)
            rows.append(q2[:, l2]); cols.append(q1[:, l1]); blks.append(-np.transpose(yb, (0, 2, 1)))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    blks = np.concatenate(blks)
    key = rows * n + cols
    ukey, where = np.unique(key, return_inverse=True)
    vals = np.zeros((ukey.shape[0], b, b))
    np.add.at(vals, where, blks)
    r_of = (ukey // n).astype(np.int64)
    col_idx = (ukey % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r_of, minlength=n))

    # Dirichlet rows and columns -> identity (pattern kept)
    cons = np.zeros((n, b), dtype=bool)
    X2, Y2 = np.arange(n2) % m2, np.arange(n2) // m2
    bnd2 = (X2 == 0) | (X2 == m2 - 1) | (Y2 == 0) | (Y2 == m2 - 1)
    X1, Y1 = np.arange(n1) % m1, np.arange(n1) // m1
    bnd1 = (X1 == 0) | (X1 == m1 - 1) | (Y1 == 0) | (Y1 == m1 - 1)
    cons[:n2][bnd2, 0:2] = True
    cons[n2:][bnd1, :] = True
    cons[0, 2] = True
    vals *= (~cons[r_of])[:, :, None]
    vals *= (~cons[col_idx])[:, None, :]
    diag = np.nonzero(r_of == col_idx)[0]
    ii, rr = np.nonzero(cons)
    vals[diag[ii], rr, rr] = 1.0
    rhs = uniform_pm1(seed, rhs_start, n * b)
    return BlockSystem(f"mhd2d_q2q1_{N}_s{seed}", n, b, row_ptr.astype(np.int32), col_idx, vals, rhs,
                       [0, 0, 0],
                       dict(kind="mhd2d_q2q1", N=N, seed=seed, nu=nu, eta=eta, tau_p=tau_p, tau_psi=tau_s, h=h,
                            n_q2=n2, n_q1=n1),
                       node_field_off=[0, n2, n])


def mhd2d_cells(N: int = 256, seed: int = 1) -> BlockSystem:
    """The 4-field system with a resistivity drawn per cell, log-uniform in
    [1e-4, 1] (the workload of the learned damping)."""
    return mhd2d(N, seed, eta_range=(1e-4, 1.0), eta_cells=True)


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

#: solver settings attached to each named workload (levels fixed where the
#: workload fixes them; otherwise coarsen while n*b > 2500, at most 10 levels)
WORKLOADS = {
    "stokes2d_32": dict(make=lambda seed=1: stokes2d(32, seed), max_levels=3, max_coarse=0,
                        restart=30, cycle="f64"),
    "mhd2d_128": dict(make=lambda seed=1: mhd2d(128, seed), max_levels=4, max_coarse=0,
                      restart=30, cycle="f64"),
    "stokes3d_64": dict(make=lambda seed=1: stokes3d(64, seed), max_levels=10, max_coarse=2500,
                        restart=50, cycle="f32"),
    "mhd2d_cells_256": dict(make=lambda seed=1: mhd2d_cells(256, seed), max_levels=10, max_coarse=2500,
                            restart=30, cycle="f32"),
}


def workload(name: str, seed: int = 1) -> BlockSystem:
    return WORKLOADS[name]["make"](seed)


def poisson_block(N: int, b: int, d: int = 2, seed: int = 1, field_of_dof=None) -> BlockSystem:
    """Q1 Laplacian (x) I_b with Dirichlet boundary: a model problem whose node
    blocks are multiples of the identity."""
    h = 1.0 / N
    dims = [N + 1] * d
    row_ptr, col_idx, pos, _, _ = _stencil_pattern(dims)
    n = int(np.prod(dims))
    vals = np.zeros((col_idx.shape[0], b, b))
    phi, dphi, _ = _q1_reference(d)
    jac = (h / 2.0) ** d
    grad = dphi * (2.0 / h)
    K = np.einsum("qla,qma->lm", grad, grad) * jac
    elem_nodes, _ = _element_nodes([N] * d)
    _scatter(vals, pos, elem_nodes, d, lambda la, lc: K[la, lc] * np.eye(b))
    cons = np.zeros((n, b), dtype=bool)
    cons[_boundary_nodes(dims), :] = True
    _apply_dirichlet(vals, row_ptr, col_idx, pos, _offset_code([0] * d), cons)
    rhs = uniform_pm1(seed, 0, n * b)
    fmap = list(field_of_dof) if field_of_dof is not None else [0] * b
    return BlockSystem(f"poisson{d}d_{N}_b{b}", n, b, row_ptr, col_idx, vals, rhs, fmap,
                       dict(kind="poisson", N=N, seed=seed, h=h))


def random_block_system(n_side: int, b: int, field_of_dof, seed: int, d: int = 2,
                        diag_shift: float = 4.0) -> BlockSystem:
    """Stencil pattern with seeded random block values and a strengthened
    diagonal: a generic nonsymmetric coupled test matrix."""
    dims = [n_side] * d
    row_ptr, col_idx, pos, _, _ = _stencil_pattern(dims)
    n = int(np.prod(dims))
    nnzb = col_idx.shape[0]
    vals = uniform_pm1(seed, 0, nnzb * b * b).reshape(nnzb, b, b)
    diag = pos[:, _offset_code([0] * d)]
    deg = np.diff(row_ptr).astype(np.float64)
    vals[diag] += (diag_shift * deg * b)[:, None, None] * np.eye(b)[None]
    rhs = uniform_pm1(seed, nnzb * b * b, n * b)
    return BlockSystem(f"random{d}d_{n_side}_b{b}_s{seed}", n, b, row_ptr, col_idx, vals,
                       rhs, list(field_of_dof), dict(kind="random", seed=seed))


# ----------------------------------------------------------------------------
# batches of independent systems
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Batch:
    """Independent systems concatenated into one block-diagonal BSR system."""

    system: BlockSystem          # the concatenation (global column indices)
    sys_node_off: np.ndarray     # int32 [nsys + 1]
    members: list                # the individual BlockSystems


def concatenate(systems) -> Batch:
    b = systems[0].b
    fm = systems[0].field_of_dof
    off = [0]
    rps, cis, vals, rhss = [], [], [], []
    blk = 0
    for s in systems:
        assert s.b == b and s.field_of_dof == fm
        rps.append(s.row_ptr[:-1].astype(np.int64) + blk)
        cis.append(s.col_idx.astype(np.int64) + off[-1])
        vals.append(s.vals)
        rhss.append(s.rhs)
        blk += s.nnzb
        off.append(off[-1] + s.n_nodes)
    row_ptr = np.concatenate(rps + [np.array([blk])]).astype(np.int32)
    col_idx = np.concatenate(cis).astype(np.int32)
    cat = BlockSystem(f"batch{len(systems)}", off[-1], b, row_ptr, col_idx, np.concatenate(vals),
                      np.concatenate(rhss), list(fm), dict(kind="batch", nsys=len(systems)))
    return Batch(cat, np.array(off, dtype=np.int32), list(systems))


def batch_sizes(nsys: int, seed: int, nmin: int = 16, nmax: int = 160) -> list:
    """Cells per side of every system, uniform integers in [nmin, nmax]."""
    u = uniform01(seed, 0, nsys)
    return [int(nmin + min(int(v * (nmax - nmin + 1)), nmax - nmin)) for v in u]


def mhd2d_batch(nsys: int = 256, seed: int = 1, nmin: int = 16, nmax: int = 160) -> Batch:
    """nsys 4-field systems of uneven sizes (cells per side uniform in
    [nmin, nmax] from `seed`), system q drawn with seed 1000 * seed + q."""
    sizes = batch_sizes(nsys, seed, nmin, nmax)
    return concatenate([mhd2d(N, 1000 * seed + q) for q, N in enumerate(sizes)])
