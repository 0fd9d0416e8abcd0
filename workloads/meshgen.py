"""Seeded synthetic tetrahedral meshes (input generation only).

This module builds the geometry the benchmarks and tests run on.  It holds
none of the time-spectral GLS arithmetic: it only produces node coordinates,
tetrahedra (4 node ids, positive orientation), boundary triangles with an
outward orientation, and an integer tag per boundary triangle.

Two families are provided:

* ``pipe``: a straight cylinder (axis z) meshed from an O-grid disk
  triangulation extruded into prisms, each prism split into 3 tetrahedra by
  the smallest-global-index rule (which keeps shared quadrilateral faces
  conforming).  The wall is exactly on r = R, which the closed-form
  Womersley and Poiseuille checks need.
* ``junction``: a Fontan-like cross of four half-cylinders (two inlets along
  +-y, two outlets along +-x) carved from a Kuhn-split Cartesian lattice,
  wall nodes projected onto the cylinder surfaces where that keeps every
  incident tetrahedron well shaped.

Boundary tags: 0 wall, 1 and 2 inlets, 3 and 4 outlets.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TAG_WALL, TAG_INLET1, TAG_INLET2, TAG_OUTLET1, TAG_OUTLET2 = 0, 1, 2, 3, 4


@dataclass
class Mesh:
    xyz: np.ndarray            # [V, 3] float64
    tets: np.ndarray           # [E, 4] int32, positive signed volume
    bfaces: np.ndarray         # [F, 3] int32, (b-a)x(c-a) points outward
    btag: np.ndarray           # [F] int32
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


# ---------------------------------------------------------------- utilities

def signed_volumes(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    p = xyz[tets]
    a = p[:, 1] - p[:, 0]
    b = p[:, 2] - p[:, 0]
    c = p[:, 3] - p[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def _orient(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    tets = tets.copy()
    neg = signed_volumes(xyz, tets) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def _compact(xyz: np.ndarray, tets: np.ndarray):
    used = np.unique(tets)
    remap = -np.ones(xyz.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return xyz[used], remap[tets]


def _morton_key(pts: np.ndarray, bits: int = 10) -> np.ndarray:
    lo = pts.min(axis=0)
    span = np.maximum(pts.max(axis=0) - lo, 1e-30)
    q = np.clip(((pts - lo) / span * ((1 << bits) - 1)).astype(np.int64), 0, (1 << bits) - 1)
    key = np.zeros(pts.shape[0], dtype=np.int64)
    for b in range(bits):
        for d in range(3):
            key |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return key


def _reorder(xyz: np.ndarray, tets: np.ndarray):
    """Space-filling-curve order for nodes and elements (memory locality)."""
    order = np.argsort(_morton_key(xyz), kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    xyz = xyz[order]
    tets = inv[tets]
    cent = xyz[tets].mean(axis=1)
    eorder = np.argsort(_morton_key(cent), kind="stable")
    return xyz, tets[eorder]


def boundary_faces(xyz: np.ndarray, tets: np.ndarray):
    """Triangles that belong to exactly one tetrahedron, oriented outward."""
    loc = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])
    opp = np.array([0, 1, 2, 3])
    faces = tets[:, loc].reshape(-1, 3)
    other = np.repeat(tets[:, opp][:, :, None], 1, axis=2).reshape(-1)
    key = np.sort(faces, axis=1)
    _, idx, cnt = np.unique(key, axis=0, return_index=True, return_counts=True)
    bidx = idx[cnt == 1]
    f = faces[bidx].copy()
    o = other[bidx]
    n = np.cross(xyz[f[:, 1]] - xyz[f[:, 0]], xyz[f[:, 2]] - xyz[f[:, 0]])
    inward = np.einsum("ij,ij->i", n, xyz[o] - xyz[f[:, 0]]) > 0
    f[inward, 1], f[inward, 2] = f[inward, 2].copy(), f[inward, 1].copy()
    return f


def _finish(xyz, tets, tagger, name, info) -> Mesh:
    xyz, tets = _compact(xyz, tets)
    tets = _orient(xyz, tets)
    xyz, tets = _reorder(xyz, tets)
    tets = _orient(xyz, tets).astype(np.int32)
    vol = signed_volumes(xyz, tets)
    if not np.all(vol > 0):
        raise RuntimeError(f"{name}: {int(np.sum(vol <= 0))} non-positive tetrahedra")
    bf = boundary_faces(xyz, tets)
    tag = tagger(xyz[bf].mean(axis=1)).astype(np.int32)
    info = dict(info)
    info.update(min_vol=float(vol.min()), max_vol=float(vol.max()))
    return Mesh(xyz=xyz, tets=tets, bfaces=bf.astype(np.int32), btag=tag, name=name, info=info)


def _jitter(xyz, tets, movable, amp, rng, tries=3):
    """Random interior displacement, reverted per node where a tet degrades."""
    v0 = signed_volumes(xyz, tets)
    node_tets = [[] for _ in range(xyz.shape[0])]
    for e, t in enumerate(tets):
        for a in t:
            node_tets[a].append(e)
    idx = np.nonzero(movable)[0]
    disp = rng.uniform(-1.0, 1.0, size=(idx.size, 3)) * amp[idx, None]
    xyz = xyz.copy()
    for k, a in enumerate(idx):
        old = xyz[a].copy()
        xyz[a] = old + disp[k]
        es = node_tets[a]
        if np.any(signed_volumes(xyz, tets[es]) < 0.3 * v0[es]):
            xyz[a] = old
    return xyz


# ---------------------------------------------------------------- pipe

def _disk_ogrid(R: float, nc: int, nr: int):
    """O-grid of the disk radius R: square core + ring; returns points, tris, wall flag."""
    a = 0.55 * R
    s = np.linspace(-a, a, nc + 1)
    X, Y = np.meshgrid(s, s, indexing="ij")
    core = np.stack([X.ravel(), Y.ravel()], axis=1)
    cid = np.arange(core.shape[0]).reshape(nc + 1, nc + 1)
    # square perimeter, counter-clockwise from (a, -a)
    per = []
    for k in range(nc):
        per.append(cid[nc, k])            # x = +a, y up
    for k in range(nc):
        per.append(cid[nc - k, nc])       # y = +a, x left
    for k in range(nc):
        per.append(cid[0, nc - k])        # x = -a, y down
    for k in range(nc):
        per.append(cid[k, 0])             # y = -a, x right
    per = np.array(per)
    P = per.size
    theta = -np.pi / 4 + 2 * np.pi * np.arange(P) / P
    circ = R * np.stack([np.cos(theta), np.sin(theta)], axis=1)
    pts = [core]
    ring_ids = [per]
    nxt = core.shape[0]
    for l in range(1, nr + 1):
        t = l / nr
        t = 1.0 - (1.0 - t) ** 1.3          # mild clustering toward the wall
        layer = (1 - t) * core[per] + t * circ
        pts.append(layer)
        ring_ids.append(np.arange(nxt, nxt + P))
        nxt += P
    pts = np.concatenate(pts, axis=0)
    quads = []
    for i in range(nc):
        for j in range(nc):
            quads.append([cid[i, j], cid[i + 1, j], cid[i + 1, j + 1], cid[i, j + 1]])
    for l in range(nr):
        r0, r1 = ring_ids[l], ring_ids[l + 1]
        for k in range(P):
            k1 = (k + 1) % P
            quads.append([r0[k], r0[k1], r1[k1], r1[k]])
    tris = []
    for q in quads:
        d1 = np.linalg.norm(pts[q[0]] - pts[q[2]])
        d2 = np.linalg.norm(pts[q[1]] - pts[q[3]])
        if d1 <= d2:
            tris += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
        else:
            tris += [[q[0], q[1], q[3]], [q[1], q[2], q[3]]]
    wall = np.zeros(pts.shape[0], dtype=bool)
    wall[ring_ids[-1]] = True
    return pts, np.array(tris), wall


def _prism_to_tets(p):
    """Split prism (p0,p1,p2 bottom; p3,p4,p5 top) by the smallest-index rule."""
    p = list(p)
    m = int(np.argmin(p))
    if m >= 3:
        p = p[3:] + p[:3]
        m -= 3
    rot = [m, (m + 1) % 3, (m + 2) % 3]
    p = [p[rot[0]], p[rot[1]], p[rot[2]], p[rot[0] + 3], p[rot[1] + 3], p[rot[2] + 3]]
    if min(p[1], p[5]) < min(p[2], p[4]):
        return [[p[0], p[1], p[2], p[5]], [p[0], p[1], p[5], p[4]], [p[0], p[4], p[5], p[3]]]
    return [[p[0], p[1], p[2], p[4]], [p[0], p[4], p[2], p[5]], [p[0], p[4], p[5], p[3]]]


def pipe(R: float = 1.0, L: float = 5.0, nc: int = 4, nr: int = 3, nz: int = 20,
         seed: int = 0, jitter: float = 0.15) -> Mesh:
    """Cylinder of radius R along z in [0, L]; inlet tag 1 at z=0, outlet tag 3 at z=L."""
    rng = np.random.default_rng(seed)
    p2, tris, wall2 = _disk_ogrid(R, nc, nr)
    n2 = p2.shape[0]
    zs = np.linspace(0.0, L, nz + 1)
    xyz = np.concatenate([np.column_stack([p2, np.full(n2, z)]) for z in zs], axis=0)
    tets = []
    for k in range(nz):
        off0, off1 = k * n2, (k + 1) * n2
        for t in tris:
            tets += _prism_to_tets([t[0] + off0, t[1] + off0, t[2] + off0,
                                    t[0] + off1, t[1] + off1, t[2] + off1])
    tets = np.array(tets, dtype=np.int64)
    tets = _orient(xyz, tets)
    layer = np.repeat(np.arange(nz + 1), n2)
    movable = (~np.tile(wall2, nz + 1)) & (layer > 0) & (layer < nz)
    h = min(L / nz, 2 * R / (nc + 2 * nr))
    xyz = _jitter(xyz, tets, movable, np.full(xyz.shape[0], jitter * h), rng)

    def tagger(c):
        tag = np.full(c.shape[0], TAG_WALL)
        tag[np.abs(c[:, 2]) < 1e-9] = TAG_INLET1
        tag[np.abs(c[:, 2] - L) < 1e-9] = TAG_OUTLET1
        return tag

    return _finish(xyz, tets, tagger, f"pipe(R={R},L={L},nc={nc},nr={nr},nz={nz},seed={seed})",
                   dict(kind="pipe", R=R, L=L, h=h))


# ---------------------------------------------------------------- junction

# arms: (axis, sign, radius); inlet along +y (1.0) and -y (0.8), outlets +-x (0.9)
JUNCTION_ARMS = (
    ("y", +1, 1.0, TAG_INLET1),
    ("y", -1, 0.8, TAG_INLET2),
    ("x", +1, 0.9, TAG_OUTLET1),
    ("x", -1, 0.9, TAG_OUTLET2),
)
_AX = {"x": 0, "y": 1, "z": 2}


def _inside_junction(p: np.ndarray, arm_len: float) -> np.ndarray:
    ins = np.zeros(p.shape[0], dtype=bool)
    for ax, sg, R, _ in JUNCTION_ARMS:
        a = _AX[ax]
        o = [d for d in range(3) if d != a]
        r2 = p[:, o[0]] ** 2 + p[:, o[1]] ** 2
        s = sg * p[:, a]
        ins |= (s >= -1e-12) & (s <= arm_len + 1e-12) & (r2 <= R * R)
    return ins


def junction(h: float = 0.123, arm_len: float = 6.0, seed: int = 1, jitter: float = 0.12,
             project: bool = True) -> Mesh:
    """Cross junction: inlets at y=+-arm_len (tags 1, 2), outlets at x=+-arm_len (tags 3, 4)."""
    rng = np.random.default_rng(seed)
    n = int(np.ceil(2 * arm_len / h))
    h = 2 * arm_len / n
    nzc = int(np.ceil(2 * 1.0 / h))
    xs = np.linspace(-arm_len, arm_len, n + 1)
    zs = -nzc * h / 2 + h * np.arange(nzc + 1)
    X, Y, Z = np.meshgrid(xs, xs, zs, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    nx, ny, nz = n + 1, n + 1, nzc + 1
    gid = np.arange(grid.shape[0]).reshape(nx, ny, nz)
    # Kuhn split of every cube: 6 monotone lattice paths from (0,0,0) to (1,1,1)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(nzc), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    cube_c = grid[gid[base[:, 0], base[:, 1], base[:, 2]]] + h / 2
    keep_cube = np.abs(cube_c[:, 0]) < arm_len + h  # all, filtered per tet below
    base = base[keep_cube]
    tets = []
    for perm in perms:
        corners = [base.copy()]
        cur = base.copy()
        for d in perm:
            cur = cur.copy()
            cur[:, d] += 1
            corners.append(cur)
        tets.append(np.stack([gid[c[:, 0], c[:, 1], c[:, 2]] for c in corners], axis=1))
    tets = np.concatenate(tets, axis=0)
    cent = grid[tets].mean(axis=1)
    tets = tets[_inside_junction(cent, arm_len)]
    xyz, tets = _compact(grid, tets)
    tets = _orient(xyz, tets)
    bf = boundary_faces(xyz, tets)
    on_plane = np.zeros(xyz.shape[0], dtype=bool)
    for ax in (0, 1):
        on_plane |= np.abs(np.abs(xyz[:, ax]) - arm_len) < 1e-9
    bnode = np.zeros(xyz.shape[0], dtype=bool)
    bnode[bf.ravel()] = True
    if project:
        xyz = _project_wall(xyz, tets, bnode, arm_len, h)
    movable = ~bnode
    xyz = _jitter(xyz, tets, movable, np.full(xyz.shape[0], jitter * h), rng)

    def tagger(c):
        tag = np.full(c.shape[0], TAG_WALL)
        tag[np.abs(c[:, 1] - arm_len) < 1e-9] = TAG_INLET1
        tag[np.abs(c[:, 1] + arm_len) < 1e-9] = TAG_INLET2
        tag[np.abs(c[:, 0] - arm_len) < 1e-9] = TAG_OUTLET1
        tag[np.abs(c[:, 0] + arm_len) < 1e-9] = TAG_OUTLET2
        return tag

    return _finish(xyz, tets, tagger, f"junction(h={h:.4f},arm={arm_len},seed={seed})",
                   dict(kind="junction", h=h, arm_len=arm_len,
                        arms=[(a, s, R, t) for a, s, R, t in JUNCTION_ARMS]))


def _project_wall(xyz, tets, bnode, arm_len, h):
    """Move wall nodes radially onto the nearest arm surface when quality allows."""
    v0 = signed_volumes(xyz, tets)
    node_tets = [[] for _ in range(xyz.shape[0])]
    for e, t in enumerate(tets):
        for a in t:
            node_tets[a].append(e)
    xyz = xyz.copy()
    for a in np.nonzero(bnode)[0]:
        p = xyz[a]
        best, bd = None, np.inf
        for ax, sg, R, _ in JUNCTION_ARMS:
            ai = _AX[ax]
            if sg * p[ai] < -1e-12:
                continue
            o = [d for d in range(3) if d != ai]
            r = np.hypot(p[o[0]], p[o[1]])
            if r < 1e-12:
                continue
            q = p.copy()
            q[o[0]] *= R / r
            q[o[1]] *= R / r
            # a candidate strictly inside another arm is not on the union's wall
            others = [arm for arm in JUNCTION_ARMS if arm[:2] != (ax, sg)]
            inside_other = False
            for ax2, sg2, R2, _ in others:
                a2 = _AX[ax2]
                o2 = [d for d in range(3) if d != a2]
                if sg2 * q[a2] > 1e-9 and q[o2[0]] ** 2 + q[o2[1]] ** 2 < (R2 - 1e-9) ** 2:
                    inside_other = True
            if inside_other:
                continue
            d = np.linalg.norm(q - p)
            if d < bd:
                best, bd = q, d
        if best is None or bd > 0.75 * h:
            continue
        old = xyz[a].copy()
        xyz[a] = best
        es = node_tets[a]
        if np.any(signed_volumes(xyz, tets[es]) < 0.15 * v0[es]):
            xyz[a] = old
    return xyz


def junction_for_tets(target_tets: int, seed: int) -> Mesh:
    """Junction whose tetrahedron count is close to ``target_tets``."""
    # tets scale like h^-3; 0.123 gives about 2.0e5 tets at arm length 6
    h = 0.123 * (2.0e5 / target_tets) ** (1.0 / 3.0)
    return junction(h=h, seed=seed)
