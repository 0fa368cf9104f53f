"""Seeded synthetic inputs: tetrahedral meshes, chemistry models and initial states.

This module generates *inputs* only.  It holds none of the method's arithmetic
(no diffusion coefficients per face, no period, no sampling): it produces the
arrays that the C ABI ``rdsplit_mesh_create`` / ``rdsplit_set_model`` /
``rdsplit_set_counts`` take, and it is shared by the tests, the benchmark and
the serial oracle's drivers.  Randomness here (vertex jitter, molecule
placement, instance sizes) comes from numpy's PCG64 with explicit seeds.

Meshes are Kuhn (Freudenthal) subdivisions of a box of cells: every cell is
split into 6 tetrahedra along its main diagonal, one per permutation of the
axes.  Cells are numbered along a Morton (Z-order) curve, as a
locality-preserving mesh numbering would be.  The paper's own meshes (a spiny dendrite, a cylinder; Sec. II.A and
Sec. III.D) are not available, so these boxes stand in for them.

Conventions (also those of the C ABI):
  * ``adj[t][f]`` is the tet across the face opposite local vertex ``f``, or
    -1 on the boundary;
  * ``area[t][f]`` is that face's area (m^2), ``dist[t][f]`` the distance
    between the centroids of ``t`` and ``adj[t][f]`` (m, 0 on the boundary);
  * ``vol[t]`` is the tet volume (m^3);
  * counts are int32 ``[T][S]`` (tet-major), canonical tet order.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

AVOGADRO = 6.02214076e23

# The 6 axis permutations of the Kuhn split, in a fixed order.
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


@dataclass
class Mesh:
    adj: np.ndarray        # int32 [T][4]
    vol: np.ndarray        # float64 [T]
    area: np.ndarray       # float64 [T][4]
    dist: np.ndarray       # float64 [T][4]
    centroid: np.ndarray   # float64 [T][3]
    shape: tuple = ()      # (nx, ny, nz) cells
    size: tuple = ()       # (Lx, Ly, Lz) metres

    @property
    def n_tets(self) -> int:
        return int(self.vol.shape[0])


@dataclass
class Model:
    """A chemistry: species diffusion constants and mass-action reactions.

    ``lhs[r][s]`` / ``rhs[r][s]`` are reactant / product stoichiometries.  Rate
    constants are SI: s^-1 (first order), M^-1 s^-1 (second order), M s^-1
    (zero order, per tet volume).  ``mask`` is ``uint8 [R][T]`` or None
    (reaction active everywhere).
    """
    D: np.ndarray                 # float64 [S] m^2/s
    lhs: np.ndarray               # int32 [R][S]
    rhs: np.ndarray               # int32 [R][S]
    k: np.ndarray                 # float64 [R]
    mask: np.ndarray | None = None
    names: list = field(default_factory=list)
    tau_scale: float = 1.0

    @property
    def n_species(self) -> int:
        return int(self.D.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.k.shape[0])


def _spread3(x: np.ndarray) -> np.ndarray:
    """Spread the low 21 bits of x so that bit b lands on bit 3b."""
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def _morton3(i, j, k) -> np.ndarray:
    return _spread3(i) | (_spread3(j) << np.uint64(1)) | (_spread3(k) << np.uint64(2))


@functools.lru_cache(maxsize=64)
def _topology(nx: int, ny: int, nz: int):
    """Vertex ids of every tet (canonical order: cells along a Morton curve,
    then the 6 permutations of each cell) and the face adjacency."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ii.reshape(-1)
    cj = jj.reshape(-1)
    ck = kk.reshape(-1)
    # cells along a Morton (Z-order) curve, so that a ball of cells is a
    # compact range of tet ids
    order = np.argsort(_morton3(ci, cj, ck), kind="stable")
    ci, cj, ck = ci[order], cj[order], ck[order]
    ncell = ci.shape[0]
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    step = np.array([sx, sy, sz], dtype=np.int64)
    v0 = ci * sx + cj * sy + ck * sz
    verts = np.empty((ncell, 6, 4), dtype=np.int64)
    for p, (a, b, c) in enumerate(_PERMS):
        verts[:, p, 0] = v0
        verts[:, p, 1] = v0 + step[a]
        verts[:, p, 2] = v0 + step[a] + step[b]
        verts[:, p, 3] = v0 + step[a] + step[b] + step[c]
    verts = verts.reshape(-1, 4)
    T = verts.shape[0]
    # faces: face f is opposite vertex f
    others = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    fv = np.sort(verts[:, others], axis=2)          # [T][4][3]
    key = (fv[:, :, 0] << 42) | (fv[:, :, 1] << 21) | fv[:, :, 2]
    key = key.reshape(-1)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    a = order[same]
    b = order[same + 1]
    adj = np.full(T * 4, -1, dtype=np.int64)
    adj[a] = b // 4
    adj[b] = a // 4
    adj = adj.reshape(T, 4).astype(np.int32)
    verts.setflags(write=False)
    adj.setflags(write=False)
    return verts, adj


def kuhn_box(nx: int, ny: int, nz: int, size=(1e-6, 1e-6, 1e-6),
             jitter: float = 0.0, mesh_seed: int = 0) -> Mesh:
    """Kuhn-split box of ``nx*ny*nz`` cells (6 tets each).

    With ``jitter > 0`` every interior vertex coordinate is displaced by a
    uniform amount in ``[-jitter*h, +jitter*h]`` (``h`` the cell spacing along
    that axis); boundary vertices stay fixed so the box faces remain planar.
    """
    verts, adj = _topology(nx, ny, nz)
    Lx, Ly, Lz = size
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    gx, gy, gz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    gx = gx.transpose(2, 1, 0).reshape(-1)
    gy = gy.transpose(2, 1, 0).reshape(-1)
    gz = gz.transpose(2, 1, 0).reshape(-1)
    X = np.stack([gx * hx, gy * hy, gz * hz], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(mesh_seed))
        interior = ((gx > 0) & (gx < nx) & (gy > 0) & (gy < ny) & (gz > 0) & (gz < nz))
        d = rng.uniform(-jitter, jitter, size=(X.shape[0], 3)) * np.array([hx, hy, hz])
        X[interior] += d[interior]
    # Unjittered Kuhn tets alternate orientation with the parity of their
    # axis permutation; a jittered tet whose orientation flipped is inverted.
    parity = np.tile(np.array([1.0, -1.0, -1.0, 1.0, 1.0, -1.0]), verts.shape[0] // 6)

    def signed_volumes(Xv):
        P = Xv[verts]
        e1 = P[:, 1] - P[:, 0]
        e2 = P[:, 2] - P[:, 0]
        e3 = P[:, 3] - P[:, 0]
        return np.einsum("ij,ij->i", e1, np.cross(e2, e3)), P

    det, P = signed_volumes(X)
    ref = np.sign(det[0] * parity[0])
    if jitter > 0.0:
        # Vertices of a tet the jitter would invert (or flatten below 5% of
        # the unjittered volume) get their displacement halved, repeatedly.
        base = hx * hy * hz
        for _ in range(60):
            bad = (det * parity * ref) < 0.05 * base
            if not bad.any():
                break
            vb = np.unique(verts[bad].reshape(-1))
            vb = vb[interior[vb]]
            d[vb] *= 0.5
            X = np.stack([gx * hx, gy * hy, gz * hz], axis=1).astype(np.float64)
            X[interior] += d[interior]
            det, P = signed_volumes(X)
    if np.any(det * parity * ref <= 0):
        raise ValueError("inverted tetrahedron in the mesh")
    vol = np.abs(det) / 6.0
    others = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    F = P[:, others]                                 # [T][4][3][3]
    cr = np.cross(F[:, :, 1] - F[:, :, 0], F[:, :, 2] - F[:, :, 0])
    area = 0.5 * np.sqrt(np.einsum("ijk,ijk->ij", cr, cr))
    cen = P.mean(axis=1)
    nbc = cen[np.maximum(adj, 0)]
    dv = nbc - cen[:, None, :]
    dist = np.sqrt(np.einsum("ijk,ijk->ij", dv, dv))
    dist[adj < 0] = 0.0
    return Mesh(adj=np.array(adj), vol=vol, area=np.ascontiguousarray(area),
                dist=np.ascontiguousarray(dist), centroid=cen, shape=(nx, ny, nz),
                size=(Lx, Ly, Lz))


def triangle_sheet(nx: int, ny: int, size=(1e-6, 1e-6), jitter: float = 0.0, mesh_seed: int = 0) -> Mesh:
    """Flat triangulated rectangle for surface diffusion (Sec. III.A:
    transfer between surface triangles): ``nx*ny`` cells, each split into two
    triangles along the diagonal from its lower-left corner; interior vertices
    jittered by up to ``jitter`` of the spacing (seeded), halved where a
    triangle would fall below 5% of its unjittered area.

    Returned in the arrays of the C ABI, read for a surface: ``vol`` is the
    triangle area (m^2), ``area[t][f]`` the length of the edge opposite local
    vertex ``f`` (m), ``dist`` the distance between triangle centroids, and
    the fourth neighbour slot is -1.  The face coefficient A/(V dist) is then
    L/(A dist) (1/m^2) and D times its sum the triangle's hop rate (1/s),
    the two-dimensional form of the same rate.
    """
    Lx, Ly = size
    hx, hy = Lx / nx, Ly / ny
    gx, gy = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    gx, gy = gx.reshape(-1), gy.reshape(-1)
    X0 = np.stack([gx * hx, gy * hy], axis=1).astype(np.float64)
    vid = lambda i, j: j * (nx + 1) + i
    tris = []
    for j in range(ny):
        for i in range(nx):
            tris.append((vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)))
            tris.append((vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)))
    tri = np.array(tris, np.int64)
    interior = (gx > 0) & (gx < nx) & (gy > 0) & (gy < ny)
    d = np.zeros_like(X0)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(mesh_seed))
        d = rng.uniform(-jitter, jitter, size=X0.shape) * np.array([hx, hy])
        d[~interior] = 0.0

    def signed_areas(X):
        P = X[tri]
        e1, e2 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
        return 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]), P

    X = X0 + d
    sa, P = signed_areas(X)
    for _ in range(60):
        bad = sa < 0.05 * 0.5 * hx * hy
        if not bad.any():
            break
        vb = np.unique(tri[bad].reshape(-1))
        d[vb] *= 0.5
        X = X0 + d
        sa, P = signed_areas(X)
    if np.any(sa <= 0):
        raise ValueError("inverted triangle in the mesh")
    T = tri.shape[0]
    # neighbours across the edge opposite each local vertex
    edge_owner = {}
    adj = -np.ones((T, 4), np.int32)
    for t in range(T):
        for f in range(3):
            a, b = sorted((int(tri[t, (f + 1) % 3]), int(tri[t, (f + 2) % 3])))
            if (a, b) in edge_owner:
                u, g = edge_owner.pop((a, b))
                adj[t, f], adj[u, g] = u, t
            else:
                edge_owner[(a, b)] = (t, f)
    area = np.zeros((T, 4))
    for f in range(3):
        e = P[:, (f + 2) % 3] - P[:, (f + 1) % 3]
        area[:, f] = np.sqrt(np.einsum("ij,ij->i", e, e))
    cen2 = P.mean(axis=1)
    cen = np.concatenate([cen2, np.zeros((T, 1))], axis=1)
    nbc = cen[np.maximum(adj, 0)]
    dv = nbc - cen[:, None, :]
    dist = np.sqrt(np.einsum("ijk,ijk->ij", dv, dv))
    dist[adj < 0] = 0.0
    return Mesh(adj=adj, vol=np.ascontiguousarray(sa), area=np.ascontiguousarray(area),
                dist=np.ascontiguousarray(dist), centroid=cen, shape=(nx, ny, 1), size=(Lx, Ly, 0.0))


def shuffle_mesh(mesh: Mesh, seed: int) -> tuple:
    """The same mesh with its tets renumbered by a seeded random permutation
    (as a mesh generator without locality might number them).  Returns
    (mesh, old_of_new): new tet i is old tet old_of_new[i]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    old = rng.permutation(mesh.n_tets)
    new_of_old = np.empty_like(old)
    new_of_old[old] = np.arange(mesh.n_tets)
    adj = mesh.adj[old]
    adj = np.where(adj >= 0, new_of_old[np.maximum(adj, 0)], -1).astype(np.int32)
    return Mesh(adj=adj, vol=mesh.vol[old].copy(), area=mesh.area[old].copy(), dist=mesh.dist[old].copy(),
                centroid=mesh.centroid[old].copy(), shape=mesh.shape, size=mesh.size), old


def cube(n: int, L: float = 1e-6, jitter: float = 0.0, mesh_seed: int = 0) -> Mesh:
    return kuhn_box(n, n, n, (L, L, L), jitter, mesh_seed)


def molecules(conc_molar: float, volume_m3: float) -> int:
    """Number of molecules of a concentration (M) in a volume (m^3), rounded."""
    return int(round(conc_molar * AVOGADRO * volume_m3 * 1e3))


def point_source(mesh: Mesh, S: int, species: int, count: int, where=None) -> np.ndarray:
    """All ``count`` molecules of ``species`` in the tet whose centroid is
    nearest ``where`` (default: box centre); ties go to the lowest tet id."""
    if where is None:
        where = np.array(mesh.size) / 2.0
    d2 = np.sum((mesh.centroid - np.asarray(where)) ** 2, axis=1)
    t = int(np.argmin(d2))
    c = np.zeros((mesh.n_tets, S), dtype=np.int32)
    c[t, species] = count
    return c


def place_by_volume(mesh: Mesh, totals, seed: int) -> np.ndarray:
    """Place ``totals[s]`` molecules of each species multinomially with
    probability proportional to tet volume."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = mesh.vol / mesh.vol.sum()
    S = len(totals)
    c = np.zeros((mesh.n_tets, S), dtype=np.int32)
    for s, n in enumerate(totals):
        if n > 0:
            c[:, s] = rng.multinomial(int(n), p)
    return c


def _reactions(S: int, spec, k):
    """Build lhs/rhs from a list of (reactants, products) index tuples."""
    R = len(spec)
    lhs = np.zeros((R, S), dtype=np.int32)
    rhs = np.zeros((R, S), dtype=np.int32)
    for r, (re, pr) in enumerate(spec):
        for s in re:
            lhs[r, s] += 1
        for s in pr:
            rhs[r, s] += 1
    return lhs, rhs, np.asarray(k, dtype=np.float64)


def diffusion_model(D=1e-12, S: int = 1) -> Model:
    Ds = np.full(S, D, dtype=np.float64)
    return Model(D=Ds, lhs=np.zeros((0, S), np.int32), rhs=np.zeros((0, S), np.int32),
                 k=np.zeros(0), names=[f"S{i}" for i in range(S)])


# --------------------------------------------------------------------------
# The five workloads (diffusion cube, reaction-diffusion cube, ensemble of
# cubes, long bar, serving requests).  Each returns plain arrays.
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mesh: Mesh
    model: Model
    counts: np.ndarray
    t_end: float
    seed: int
    notes: dict = field(default_factory=dict)


def diffusion_cube(n: int = 8, L: float = 1e-6, jitter: float = 0.0, mesh_seed: int = 0,
                   n0: int = 6000, t_end: float = 0.1, seed: int = 1, D: float = 1e-12) -> Workload:
    """1-species diffusion from a point source in a Kuhn cube (n^3*6 tets)."""
    mesh = cube(n, L, jitter, mesh_seed)
    model = diffusion_model(D)
    counts = point_source(mesh, 1, 0, n0)
    return Workload(f"diffusion_cube_n{n}", mesh, model, counts, t_end, seed,
                    {"n": n, "L_m": L, "jitter": jitter, "mesh_seed": mesh_seed, "n0": n0})


def config_diffusion_3072() -> Workload:
    """8^3*6 = 3,072-tet unjittered 1 um cube, D=1e-12, 6,000 molecules at the
    centre tet, t_end = 0.1 s, seed 1."""
    w = diffusion_cube(8, 1e-6, 0.0, 0, 6000, 0.1, 1)
    w.name = "diffusion_cube_3072"
    return w


def abc_model(mask=None) -> Model:
    """A+B->C (1e6 /M/s), C->A+B (1 /s), A->0 (0.5 /s); D = 1.0, 0.5, 0.2 um^2/s."""
    S = 3
    lhs, rhs, k = _reactions(S, [((0, 1), (2,)), ((2,), (0, 1)), ((0,), ())], [1e6, 1.0, 0.5])
    return Model(D=np.array([1.0e-12, 0.5e-12, 0.2e-12]), lhs=lhs, rhs=rhs, k=k,
                 mask=mask, names=["A", "B", "C"])


def config_reaction_diffusion_48k(mesh_seed: int = 2, place_seed: int = 3) -> Workload:
    """20^3*6 = 48,000-tet 2 um cube, +-20% jitter; A,B,C chemistry; A=B=10 uM
    placed multinomially by volume; t_end = 0.5 s; seed 1."""
    L = 2e-6
    mesh = cube(20, L, 0.2, mesh_seed)
    model = abc_model()
    n = molecules(10e-6, L ** 3)
    counts = place_by_volume(mesh, [n, n, 0], place_seed)
    return Workload("reaction_diffusion_cube_48000", mesh, model, counts, 0.5, 1,
                    {"n": 20, "L_m": L, "jitter": 0.2, "mesh_seed": mesh_seed,
                     "place_seed": place_seed, "A0=B0": n})


def ensemble_sizes(n_instances: int = 512, lo: int = 6, hi: int = 40, seed: int = 3) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_instances)


def ensemble_instance(i: int, n: int, t_end: float = 0.1) -> Workload:
    """Instance ``i`` of the batched ensemble: jittered 1 um n^3*6 cube (mesh
    seed 1000+i), 1 species D=1e-12, 6,000 molecules at the centre tet,
    simulation seed i+1."""
    w = diffusion_cube(int(n), 1e-6, 0.2, 1000 + i, 6000, t_end, i + 1)
    w.name = f"ensemble_{i}_n{n}"
    return w


def bar_model(mesh: Mesh) -> Model:
    """8 species, 14 reactions on the long bar.

    Species: X, Y, Z (free), B1, B2 (buffers), XB1, YB2, ZB2 (complexes).
    Reactions: zero-order influx of X, Y, Z (1e-3 M/s, only in tets whose
    centroid has z < 1% of the bar length); X+B1<->XB1 (1e7 /M/s, 10 /s),
    Y+B2<->YB2 (3e7 /M/s, 100 /s), Z+B2<->ZB2 (1e8 /M/s, 1000 /s); first-order
    pumps X,Y,Z -> 0 (100 /s); X+Y -> Z (1e6 /M/s) and Z -> X+Y (1 /s).
    """
    S = 8
    X, Y, Z, B1, B2, XB1, YB2, ZB2 = range(S)
    spec = [((), (X,)), ((), (Y,)), ((), (Z,)),
            ((X, B1), (XB1,)), ((XB1,), (X, B1)),
            ((Y, B2), (YB2,)), ((YB2,), (Y, B2)),
            ((Z, B2), (ZB2,)), ((ZB2,), (Z, B2)),
            ((X,), ()), ((Y,), ()), ((Z,), ()),
            ((X, Y), (Z,)), ((Z,), (X, Y))]
    k = [1e-3, 1e-3, 1e-3, 1e7, 10.0, 3e7, 100.0, 1e8, 1000.0, 100.0, 100.0, 100.0, 1e6, 1.0]
    lhs, rhs, k = _reactions(S, spec, k)
    R = len(k)
    zlim = 0.01 * mesh.size[2]
    influx = (mesh.centroid[:, 2] < zlim).astype(np.uint8)
    mask = np.ones((R, mesh.n_tets), dtype=np.uint8)
    mask[0:3] = influx
    D = np.array([0.5, 0.3, 0.2, 0.05, 0.1, 0.05, 0.08, 0.1]) * 1e-12
    return Model(D=D, lhs=lhs, rhs=rhs, k=k, mask=mask,
                 names=["X", "Y", "Z", "B1", "B2", "XB1", "YB2", "ZB2"])


def config_bar(nx: int = 20, ny: int = 20, nz: int = 1000, mesh_seed: int = 4,
               place_seed: int = 5, t_end: float = 0.01) -> Workload:
    """20x20x1000 cells *6 = 2.4M tets, 1x1x50 um bar, +-20% jitter; 8 species,
    14 reactions; free species at 0.1 uM, buffers at 50 uM; t_end = 10 ms."""
    h = 0.05e-6
    size = (nx * h, ny * h, nz * h)
    mesh = kuhn_box(nx, ny, nz, size, 0.2, mesh_seed)
    model = bar_model(mesh)
    Vtot = size[0] * size[1] * size[2]
    free = molecules(0.1e-6, Vtot)
    buf = molecules(50e-6, Vtot)
    counts = place_by_volume(mesh, [free, free, free, buf, buf, 0, 0, 0], place_seed)
    return Workload(f"bar_{nx}x{ny}x{nz}", mesh, model, counts, t_end, 1,
                    {"cells": [nx, ny, nz], "h_m": h, "jitter": 0.2,
                     "mesh_seed": mesh_seed, "place_seed": place_seed})


def random_model(mesh: Mesh, S: int, rng: np.random.Generator) -> Model:
    """Random chemistry in the style of the bar model: S species with D in
    [0.05, 0.5] um^2/s; a zero-order influx of species 0 in the first 1% of
    the box along z; first-order conversions s -> s+1; reversible bindings
    s + (s+1) <-> (s+2); first-order removal of the last species."""
    D = rng.uniform(0.05, 0.5, size=S) * 1e-12
    spec, k = [((), (0,))], [1e-3]
    for s in range(S - 1):
        spec.append(((s,), (s + 1,)))
        k.append(float(10 ** rng.uniform(0, 2)))
    for s in range(S - 2):
        spec.append(((s, s + 1), (s + 2,)))
        k.append(float(10 ** rng.uniform(6, 8)))
        spec.append(((s + 2,), (s, s + 1)))
        k.append(float(10 ** rng.uniform(1, 3)))
    spec.append(((S - 1,), ()))
    k.append(100.0)
    lhs, rhs, kk = _reactions(S, spec, k)
    R = len(kk)
    zlim = 0.01 * mesh.size[2]
    mask = np.ones((R, mesh.n_tets), dtype=np.uint8)
    mask[0] = (mesh.centroid[:, 2] < zlim).astype(np.uint8)
    return Model(D=D, lhs=lhs, rhs=rhs, k=kk, mask=mask, names=[f"S{i}" for i in range(S)])


@dataclass
class Request:
    """One serving request; ``workload()`` builds its mesh and model on demand."""
    rid: int
    arrival: float
    n: int
    S: int
    t_end: float
    model_seed: int
    h: float = 0.05e-6

    def workload(self) -> Workload:
        L = self.n * self.h
        mesh = cube(self.n, L, 0.2, 5000 + self.rid)
        rng = np.random.Generator(np.random.PCG64(self.model_seed))
        model = random_model(mesh, self.S, rng)
        free = molecules(1e-6, L ** 3)
        counts = place_by_volume(mesh, [free] * self.S, 7000 + self.rid)
        return Workload(f"request_{self.rid}_n{self.n}_S{self.S}", mesh, model, counts, self.t_end,
                        100 + self.rid, {"n": self.n, "S": self.S, "h_m": self.h})

    @property
    def n_tets(self) -> int:
        return 6 * self.n ** 3


def serving_requests(n_requests: int, rate: float = 200.0, seed: int = 5,
                     n_lo: int = 6, n_hi: int = 60, tmin: float = 1e-3, tmax: float = 50e-3,
                     h: float = 0.05e-6) -> list:
    """Poisson arrivals at ``rate``/s; each request a jittered n^3*6 cube with
    n log-uniform in [n_lo, n_hi] and cell size ``h``, 1-8 species, random
    chemistry (``random_model``), t_end uniform in [tmin, tmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        S = int(rng.integers(1, 9))
        t_end = float(rng.uniform(tmin, tmax))
        out.append(Request(i, t, n, S, t_end, 9000 + i, h))
    return out
