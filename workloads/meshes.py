"""Structured and mapped simplex meshes (coordinates + cells only).

Every generator returns ``(coords, cells)``: ``coords`` is a float64 array of
shape (n_nodes, dim) in centimetres and ``cells`` an int64 array of shape
(n_cells, dim + 1) of node indices.  Node numbering is lexicographic with x
fastest, so a structured grid's stiffness matrix is banded.

Meshing choices the paper leaves open (its experiments only name the domain
and the mesh size, Sec. 5.2-5.3):
  * 2-D: every grid square is split along its (i, j) -> (i+1, j+1) diagonal.
  * 3-D: every grid cube is split into the 6 Kuhn tetrahedra that share its
    (0,0,0) -> (1,1,1) main diagonal.
Both choices are translation invariant in index space, hence conforming.
"""

from __future__ import annotations

import numpy as np

from .fields import splitmix64, u01


def line_mesh(n: int, length: float):
    """Uniform 1-D P1 mesh of [0, length] with ``n`` nodes."""
    if n < 2:
        raise ValueError("a line mesh needs at least 2 nodes")
    x = np.linspace(0.0, length, n)
    cells = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int64)
    return x[:, None].copy(), cells


def square_tri_mesh(nx: int, ny: int, lx: float, ly: float):
    """Right-diagonal triangulation of [0,lx] x [0,ly] with nx x ny nodes."""
    if nx < 2 or ny < 2:
        raise ValueError("need at least 2 nodes per axis")
    xs = np.linspace(0.0, lx, nx)
    ys = np.linspace(0.0, ly, ny)
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # shape (ny, nx), x fastest
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    a = (j * nx + i).ravel()
    b = a + 1
    c = a + nx + 1
    d = a + nx
    cells = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return coords, cells.astype(np.int64)


# The 6 permutations of the axes; each gives one Kuhn tetrahedron as the
# monotone lattice path origin -> +e_p0 -> +e_p1 -> +e_p2.
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _kuhn_cells(node_id, ni, nj, nk, wrap_k=False):
    """Kuhn tetrahedra of an (ni-1) x (nj-1) x (nk-1) grid of cubes.

    ``node_id(i, j, k)`` maps integer lattice arrays to node indices.  With
    ``wrap_k`` the third axis is periodic (nk cubes instead of nk-1).
    """
    kc = nk if wrap_k else nk - 1
    I, J, K = np.meshgrid(np.arange(ni - 1), np.arange(nj - 1), np.arange(kc), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    out = []
    for p in _PERMS:
        verts = []
        off = [0, 0, 0]
        verts.append(node_id(I, J, K))
        for ax in p:
            off[ax] += 1
            kk = K + off[2]
            if wrap_k:
                kk = kk % nk
            verts.append(node_id(I + off[0], J + off[1], kk))
        out.append(np.stack(verts, axis=1))
    return np.concatenate(out, axis=0)


def slab_tet_mesh(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float):
    """Kuhn 6-tet mesh of the box [0,lx] x [0,ly] x [0,lz]."""
    if min(nx, ny, nz) < 2:
        raise ValueError("need at least 2 nodes per axis")
    xs = np.linspace(0.0, lx, nx)
    ys = np.linspace(0.0, ly, ny)
    zs = np.linspace(0.0, lz, nz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")  # (nz, ny, nx), x fastest
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def nid(i, j, k):  # i along x, j along y, k along z
        return (k * ny + j) * nx + i

    cells = _kuhn_cells(nid, nx, ny, nz)
    return coords, cells.astype(np.int64)


def _signed_vol6(coords, cells):
    p = coords[cells]
    e1 = p[:, 1] - p[:, 0]
    e2 = p[:, 2] - p[:, 0]
    e3 = p[:, 3] - p[:, 0]
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3))


def shell_tet_mesh(nr: int = 32, nuv: int = 362, *, rs_in: float = 1.8, rl_in: float = 4.3,
                   thick: float = 0.7, z_top: float = 2.0, jitter: float = 0.2, seed: int = 2,
                   return_param: bool = False):
    """Truncated prolate-ellipsoidal shell ("ventricle-like"), Kuhn tets.

    A structured box grid (r, u, v) in [0,1] x [-1,1]^2 is mapped onto the shell
    without a pole: the square (u, v) goes into the unit disk by the blended
    elliptical map x = c u sqrt(1 - v^2/4), y = c v sqrt(1 - u^2/4),
    c = sqrt(2/3) (corners on the unit circle, edge midpoints at radius c; a
    map that puts the whole square boundary on the circle flattens the corner
    cells).  The radius rho and angle phi give the polar angle
    theta = pi - rho (pi - theta_top(r)) from the apex (theta = pi), with
    theta_top(r) = arccos(z_top/Rl(r)), so the corners reach the plane
    z = z_top and the rim dips below it between them; then
        x = Rs(r) sin(theta) cos(phi), y = Rs(r) sin(theta) sin(phi),
        z = Rl(r) cos(theta),  Rs = rs_in + thick*r,  Rl = rl_in + thick*r.
    Interior nodes (not on r = 0, r = 1 or the truncation rim) are jittered by
    U(-jitter, jitter) of the local parametric spacing in each parametric
    direction (seeded counter-based generator); a node's jitter is halved
    while any of its tetrahedra inverts or degenerates.
    """
    r = np.linspace(0.0, 1.0, nr)
    uv = np.linspace(-1.0, 1.0, nuv)
    I, J, K = np.meshgrid(np.arange(nr), np.arange(nuv), np.arange(nuv), indexing="ij")
    n_nodes = nr * nuv * nuv

    def nid(i, j, k):
        return (np.asarray(i) * nuv + np.asarray(j)) * nuv + np.asarray(k)

    pr = r[I].ravel().astype(np.float64)
    pu = uv[J].ravel().astype(np.float64)
    pv = uv[K].ravel().astype(np.float64)
    interior = ((I > 0) & (I < nr - 1) & (J > 0) & (J < nuv - 1) & (K > 0) & (K < nuv - 1)).ravel()
    cells = _kuhn_cells(nid, nr, nuv, nuv)

    def to_xyz(pr_, pu_, pv_):
        pu_ = np.clip(pu_, -1.0, 1.0)
        pv_ = np.clip(pv_, -1.0, 1.0)
        c = np.sqrt(2.0 / 3.0)
        xd = c * pu_ * np.sqrt(1.0 - 0.25 * pv_ * pv_)
        yd = c * pv_ * np.sqrt(1.0 - 0.25 * pu_ * pu_)
        rho = np.minimum(np.hypot(xd, yd), 1.0)
        ph = np.arctan2(yd, xd)
        rs = rs_in + thick * pr_
        rl = rl_in + thick * pr_
        th_top = np.arccos(z_top / rl)
        th = np.pi - rho * (np.pi - th_top)
        return np.stack([rs * np.sin(th) * np.cos(ph), rs * np.sin(th) * np.sin(ph), rl * np.cos(th)], axis=1)

    xyz0 = to_xyz(pr, pu, pv)
    vol0 = _signed_vol6(xyz0, cells)
    sign0 = np.sign(vol0)
    if np.any(sign0 == 0):
        raise RuntimeError("degenerate tetrahedron in the unjittered shell")
    idx = np.arange(n_nodes, dtype=np.uint64)
    scale = np.where(interior, jitter, 0.0)
    jr = u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(0), idx)) * 2 - 1
    ju = u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(1), idx)) * 2 - 1
    jv = u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(2), idx)) * 2 - 1
    dr = 1.0 / (nr - 1)
    duv = 2.0 / (nuv - 1)
    for _ in range(12):
        xyz = to_xyz(pr + scale * jr * dr, pu + scale * ju * duv, pv + scale * jv * duv)
        vol = _signed_vol6(xyz, cells)
        bad = (np.sign(vol) != sign0) | (np.abs(vol) < 1e-2 * np.abs(vol0))
        if not np.any(bad):
            break
        scale[np.unique(cells[bad].ravel())] *= 0.5
    else:
        raise RuntimeError("shell jitter did not converge")
    if return_param:
        return xyz, cells.astype(np.int64), (pr, rs_in, rl_in, thick, z_top)
    return xyz, cells.astype(np.int64)
