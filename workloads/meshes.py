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


def shell_tet_mesh(nr: int = 32, ntheta: int = 256, nphi: int = 512, *,
                   rs_in: float = 1.8, rl_in: float = 4.3, thick: float = 0.7,
                   z_top: float = 2.0, jitter: float = 0.2, seed: int = 2,
                   return_param: bool = False):
    """Truncated prolate-ellipsoidal shell ("ventricle-like"), Kuhn tets.

    Parametric grid (r, theta, phi) in [0,1] x [theta_top(r), pi] x [0, 2pi):
        x = Rs(r) sin(theta) cos(phi), y = Rs(r) sin(theta) sin(phi),
        z = Rl(r) cos(theta),  Rs = rs_in + thick*r,  Rl = rl_in + thick*r,
    with theta_top(r) = arccos(z_top / Rl(r)) (the base plane z = z_top).
    The theta = pi ring of every r collapses to one apex node; tetrahedra with
    a repeated vertex are dropped.  Interior nodes (not on r=0, r=1, the base
    or the apex) are jittered by U(-jitter, jitter) of the local parametric
    spacing in each parametric direction (seeded counter-based generator);
    a node's jitter is halved while any of its tetrahedra inverts.
    """
    nt = ntheta
    r = np.linspace(0.0, 1.0, nr)
    # node ids: rings j < nt-1 are full, j = nt-1 is the apex (one per r)
    n_ring = (nt - 1) * nphi
    n_nodes = nr * (n_ring + 1)

    def nid(i, j, k):
        i = np.asarray(i)
        j = np.asarray(j)
        k = np.asarray(k)
        base = i * (n_ring + 1)
        return np.where(j >= nt - 1, base + n_ring, base + j * nphi + k)

    # parametric coordinates of every node (apex entries set separately)
    I, J, K = np.meshgrid(np.arange(nr), np.arange(nt - 1), np.arange(nphi), indexing="ij")
    rr = r[I].astype(np.float64)
    tt = J.astype(np.float64)  # theta index (fractional after jitter)
    pp = K.astype(np.float64)
    ids = nid(I, J, K).ravel()
    pr = np.empty(n_nodes)
    pt = np.empty(n_nodes)
    pph = np.empty(n_nodes)
    pr[ids] = rr.ravel()
    pt[ids] = tt.ravel()
    pph[ids] = pp.ravel()
    apex = np.arange(nr) * (n_ring + 1) + n_ring
    pr[apex] = r
    pt[apex] = nt - 1
    pph[apex] = 0.0

    interior = np.zeros(n_nodes, dtype=bool)
    inner_mask = (I > 0) & (I < nr - 1) & (J > 0)
    interior[ids[inner_mask.ravel()]] = True

    cells = _kuhn_cells(nid, nr, nt, nphi, wrap_k=True)
    # drop degenerate tetrahedra (repeated vertex at the apex)
    srt = np.sort(cells, axis=1)
    keep = np.all(srt[:, 1:] != srt[:, :-1], axis=1)
    cells = cells[keep]

    def to_xyz(pr_, pt_, pph_):
        rs = rs_in + thick * pr_
        rl = rl_in + thick * pr_
        th_top = np.arccos(z_top / rl)
        th = th_top + (np.pi - th_top) * (pt_ / (nt - 1))
        ph = 2.0 * np.pi * pph_ / nphi
        return np.stack([rs * np.sin(th) * np.cos(ph),
                         rs * np.sin(th) * np.sin(ph),
                         rl * np.cos(th)], axis=1)

    xyz0 = to_xyz(pr, pt, pph)
    xyz0[apex, 0] = 0.0
    xyz0[apex, 1] = 0.0
    sign0 = np.sign(_signed_vol6(xyz0, cells))
    if np.any(sign0 == 0):
        raise RuntimeError("degenerate tetrahedron in the unjittered shell")

    # seeded jitter: three counter streams, one per parametric direction
    idx = np.arange(n_nodes, dtype=np.uint64)
    scale = np.where(interior, jitter, 0.0)
    jr = (u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(0), idx)) * 2 - 1)
    jt = (u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(1), idx)) * 2 - 1)
    jp = (u01(splitmix64(np.uint64(seed) * np.uint64(3) + np.uint64(2), idx)) * 2 - 1)
    dr = 1.0 / (nr - 1)
    for _ in range(12):
        xyz = to_xyz(pr + scale * jr * dr, pt + scale * jt, pph + scale * jp)
        xyz[apex, 0] = 0.0
        xyz[apex, 1] = 0.0
        vol = _signed_vol6(xyz, cells)
        bad = (np.sign(vol) != sign0) | (np.abs(vol) < 1e-3 * np.abs(_signed_vol6(xyz0, cells)))
        if not np.any(bad):
            break
        bad_nodes = np.unique(cells[bad].ravel())
        scale[bad_nodes] *= 0.5
    else:
        raise RuntimeError("shell jitter did not converge")
    if return_param:
        return xyz, cells.astype(np.int64), (pr, pt, pph, rs_in, rl_in, thick, z_top, nt, nphi)
    return xyz, cells.astype(np.int64)
