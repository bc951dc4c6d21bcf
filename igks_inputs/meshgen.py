"""Seeded synthetic mesh generators for 2D unstructured hybrid (quad + triangle) meshes.

This module is an INPUT GENERATOR shared by the CPU oracle tests and the CUDA path.
It holds only topology and node placement: no flux, gradient, limiter, boundary-state
or sweep arithmetic of the gas-kinetic method lives here.

A mesh is returned as plain numpy arrays in the face/cell layout the C ABI takes:

    xy          float64 [n_nodes, 2]     node coordinates
    cell_ptr    int32   [n_cells + 1]    CSR offsets into cell_nodes
    cell_nodes  int32   [...]            counter-clockwise node lists, one per cell
    face_nodes  int32   [n_faces, 2]     (a, b): a->b runs counter-clockwise around the
                                         left cell, so the right-hand normal of a->b
                                         points out of the left cell
    face_cells  int32   [n_faces, 2]     (left, right); right = -1 on a boundary face
    face_bc     int32   [n_faces]        0 interior, 1 free stream, 2 symmetry, 3 wall, 4 outflow,
                                         5 moving wall

Faces are numbered in the order they are first met while scanning cells in order and,
inside a cell, its edges in counter-clockwise order. Cells keep the generator's order;
that order is the sweep order of the LU-SGS method (Eq. 20, j < i by index).

The configurations follow the paper's workloads in kind and size (Section III: laminar
and turbulent flat plates on hybrid meshes of 1e4-6e4 cells, an airfoil with body-fitted
quad layers and triangles outside), with synthetic geometry since no mesh of the paper
is available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_INTERIOR, BC_FARFIELD, BC_SYMMETRY, BC_WALL, BC_OUTFLOW, BC_MOVING_WALL = 0, 1, 2, 3, 4, 5


@dataclass
class Mesh:
    xy: np.ndarray
    cell_ptr: np.ndarray
    cell_nodes: np.ndarray
    face_nodes: np.ndarray
    face_cells: np.ndarray
    face_bc: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cell_ptr.shape[0] - 1)

    @property
    def n_faces(self) -> int:
        return int(self.face_nodes.shape[0])

    def cell_node_list(self, c: int) -> np.ndarray:
        return self.cell_nodes[self.cell_ptr[c]:self.cell_ptr[c + 1]]

    def renumbered(self, perm: np.ndarray) -> "Mesh":
        """Return the same mesh with cell k of the result = cell perm[k] of this one.

        Faces are rebuilt from the renumbered cells, so face order and orientation follow
        the same rule as every generated mesh."""
        cells = [self.cell_node_list(int(c)) for c in perm]
        m = build_mesh(self.xy, cells, _bc_from_faces(self), name=self.name)
        m.meta = dict(self.meta)
        return m


def _bc_from_faces(mesh: Mesh):
    """Boundary tags of an existing mesh, keyed by the sorted node pair."""
    table = {}
    for f in range(mesh.n_faces):
        if mesh.face_cells[f, 1] < 0:
            a, b = int(mesh.face_nodes[f, 0]), int(mesh.face_nodes[f, 1])
            table[(min(a, b), max(a, b))] = int(mesh.face_bc[f])
    return lambda a, b, xm, ym: table[(min(a, b), max(a, b))]


def build_mesh(xy: np.ndarray, cells, bc_of, name: str = "") -> Mesh:
    """Build the face list of a mesh given its nodes and CCW cell node lists.

    bc_of(a, b, xm, ym) returns the boundary tag of a boundary edge a->b with midpoint
    (xm, ym)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    sizes = np.fromiter((len(n) for n in cells), dtype=np.int64, count=len(cells))
    ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    flat = np.concatenate([np.asarray(n, dtype=np.int64) for n in cells]) if cells else np.zeros(0, np.int64)
    # directed edges a -> b of every cell, in cell order and CCW order inside a cell
    owner = np.repeat(np.arange(len(cells), dtype=np.int64), sizes)
    pos = np.arange(flat.shape[0], dtype=np.int64) - ptr[owner]
    nxt = np.where(pos + 1 < sizes[owner], np.arange(flat.shape[0]) + 1, ptr[owner])
    ea, eb = flat, flat[nxt]
    key = np.minimum(ea, eb) * (xy.shape[0] + 1) + np.maximum(ea, eb)
    # faces numbered by first appearance of their edge
    uniq, first, inv, cnt = np.unique(key, return_index=True, return_inverse=True, return_counts=True)
    if np.any(cnt > 2):
        raise ValueError("an edge is shared by more than two cells")
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.shape[0])
    fid = rank[inv]                                   # face of every directed edge
    nf = uniq.shape[0]
    face_nodes = np.empty((nf, 2), dtype=np.int64)
    face_cells = np.full((nf, 2), -1, dtype=np.int64)
    fe = first[order]                                 # first occurrence of each face
    face_nodes[:, 0], face_nodes[:, 1] = ea[fe], eb[fe]
    face_cells[:, 0] = owner[fe]
    second = np.ones(flat.shape[0], dtype=bool)
    second[fe] = False
    sec = np.nonzero(second)[0]
    if np.any((ea[sec] != face_nodes[fid[sec], 1]) | (eb[sec] != face_nodes[fid[sec], 0])):
        raise ValueError("inconsistent orientation between two cells sharing an edge")
    face_cells[fid[sec], 1] = owner[sec]
    face_nodes = face_nodes.astype(np.int32)
    face_cells = face_cells.astype(np.int32)
    face_bc = np.zeros(nf, dtype=np.int32)
    for f in range(face_nodes.shape[0]):
        if face_cells[f, 1] < 0:
            a, b = face_nodes[f]
            xm = 0.5 * (xy[a, 0] + xy[b, 0])
            ym = 0.5 * (xy[a, 1] + xy[b, 1])
            face_bc[f] = bc_of(int(a), int(b), xm, ym)
    m = Mesh(xy=xy, cell_ptr=ptr.astype(np.int32), cell_nodes=flat.astype(np.int32),
             face_nodes=face_nodes, face_cells=face_cells, face_bc=face_bc, name=name)
    _check_ccw(m)
    return m


def _check_ccw(m: Mesh) -> None:
    """Every cell must be a simple polygon listed counter-clockwise (signed area > 0)."""
    ptr = m.cell_ptr.astype(np.int64)
    sizes = np.diff(ptr)
    owner = np.repeat(np.arange(m.n_cells), sizes)
    idx = np.arange(m.cell_nodes.shape[0])
    nxt = np.where(idx + 1 < ptr[owner + 1], idx + 1, ptr[owner])
    p, q = m.cell_nodes, m.cell_nodes[nxt]
    cross = m.xy[p, 0] * m.xy[q, 1] - m.xy[q, 0] * m.xy[p, 1]
    area = 0.5 * np.add.reduceat(cross, ptr[:-1]) if m.n_cells else np.zeros(0)
    bad = np.nonzero(~(area > 0.0))[0]
    if bad.size:
        raise ValueError(f"{m.name}: cell {bad[0]} has non-positive signed area {area[bad[0]]}")


# --------------------------------------------------------------------------------------
# spacing helpers
# --------------------------------------------------------------------------------------

def geometric_levels(first: float, ratio: float, n: int) -> np.ndarray:
    """n+1 monotone coordinates starting at 0 with first spacing `first`, growth `ratio`."""
    h = first * ratio ** np.arange(n)
    return np.concatenate([[0.0], np.cumsum(h)])


def _solve_ratio(first: float, total: float, n: int) -> float:
    """Growth ratio r with first*(r^n-1)/(r-1) = total (bisection)."""
    if abs(first * n - total) < 1e-15 * total:
        return 1.0
    lo, hi = (1.0 + 1e-12, 10.0) if first * n < total else (1e-6, 1.0 - 1e-12)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = first * (mid ** n - 1.0) / (mid - 1.0)
        if (s < total) == (first * n < total):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# --------------------------------------------------------------------------------------
# flat plate meshes (laminar and turbulent plate workloads)
# --------------------------------------------------------------------------------------

def _plate_bc(x0_wall: float = 0.0, xmin: float = -0.5, xmax: float = 1.0, ymax: float = 1.0):
    tol = 1e-12

    # as the paper's flat plates: free stream at the inflow (left) boundary, the
    # Riemann-invariant outflow condition on the upper and outflow boundaries
    def bc(a, b, xm, ym):
        if abs(ym) < tol:
            return BC_WALL if xm >= x0_wall else BC_SYMMETRY
        return BC_FARFIELD if abs(xm - xmin) < tol else BC_OUTFLOW
    return bc


def flat_plate_quads(nx: int = 64, ny: int = 32, ratio: float = 1.1,
                     xmin: float = -0.5, xmax: float = 1.0, height: float = 1.0,
                     first: float | None = None, name: str = "plate_quads") -> Mesh:
    """Structured nx x ny quad mesh of the laminar flat plate, stored unstructured.

    x uniform on [xmin, xmax]; y geometric with `ratio` on [0, height] (or with the
    given first spacing, the ratio then solved so the layer reaches `height`).
    Wall on y = 0 for x >= 0, symmetry on y = 0 for x < 0, free stream at the inflow (left),
    outflow on the upper and right boundaries."""
    xs = np.linspace(xmin, xmax, nx + 1)
    if first is None:
        first = height * (ratio - 1.0) / (ratio ** ny - 1.0) if ratio != 1.0 else height / ny
    else:
        ratio = _solve_ratio(first, height, ny)
    ys = geometric_levels(first, ratio, ny)
    ys *= height / ys[-1]
    ys[-1] = height
    X, Y = np.meshgrid(xs, ys)  # [ny+1, nx+1]
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    nid = lambda i, j: j * (nx + 1) + i
    cells = []
    for j in range(ny):
        for i in range(nx):
            cells.append([nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)])
    m = build_mesh(xy, cells, _plate_bc(xmin=xmin), name=name)
    m.meta = dict(kind="plate", nx=nx, ny=ny, first=float(first), ratio=float(ratio))
    return m


def flat_plate_hybrid(nx: int = 128, nq: int = 64, ntri_rows: int = 48, first: float = 1e-6,
                      ratio: float = 1.15, xmin: float = -0.5, xmax: float = 1.0,
                      height: float = 1.0, jitter: float = 0.25, seed: int = 1,
                      name: str = "plate_hybrid") -> Mesh:
    """Hybrid flat plate mesh: an nx x nq quad boundary layer (first spacing `first`,
    growth `ratio`) topped by a jittered (nx+1) x (ntri_rows+1)-point lattice up to
    `height`, each lattice cell split along a seeded-random diagonal into two triangles.

    The lattice's bottom row is the quad layer's top row. Lattice rows grow
    geometrically from 1.15 x the last quad height; interior lattice points are moved
    uniformly by up to +-jitter of the local spacing; boundary points stay in place."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(xmin, xmax, nx + 1)
    yq = geometric_levels(first, ratio, nq)
    top_q = yq[-1]
    h0 = (yq[-1] - yq[-2]) * ratio
    r2 = _solve_ratio(h0, height - top_q, ntri_rows)
    yt = top_q + geometric_levels(h0, r2, ntri_rows)
    yt[-1] = height
    # node rows: quad rows 0..nq, then lattice rows 1..ntri_rows (row 0 shared)
    ys_all = np.concatenate([yq, yt[1:]])
    nrows = ys_all.shape[0]
    X, Y = np.meshgrid(xs, ys_all)
    X = X.copy()
    Y = Y.copy()
    dx = xs[1] - xs[0]
    for r in range(nq + 1, nrows - 1):
        dy_lo = ys_all[r] - ys_all[r - 1]
        dy_hi = ys_all[r + 1] - ys_all[r]
        for i in range(1, nx):
            X[r, i] += jitter * dx * rng.uniform(-1.0, 1.0)
            Y[r, i] += jitter * min(dy_lo, dy_hi) * rng.uniform(-1.0, 1.0)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    nid = lambda i, r: r * (nx + 1) + i
    cells = []
    for r in range(nq):
        for i in range(nx):
            cells.append([nid(i, r), nid(i + 1, r), nid(i + 1, r + 1), nid(i, r + 1)])
    diag = rng.integers(0, 2, size=(ntri_rows, nx))
    for rr in range(ntri_rows):
        r = nq + rr
        for i in range(nx):
            a, b, c, d = nid(i, r), nid(i + 1, r), nid(i + 1, r + 1), nid(i, r + 1)
            if diag[rr, i] == 0:   # split along a-c
                cells.append([a, b, c])
                cells.append([a, c, d])
            else:                  # split along b-d
                cells.append([a, b, d])
                cells.append([b, c, d])
    m = build_mesh(xy, cells, _plate_bc(xmin=xmin), name=name)
    m.meta = dict(kind="plate_hybrid", nx=nx, nq=nq, ntri_rows=ntri_rows, first=first,
                  ratio=ratio, seed=seed)
    return m


# --------------------------------------------------------------------------------------
# NACA 4-digit O-mesh (airfoil workloads)
# --------------------------------------------------------------------------------------

def naca4_surface(m: float, p: float, t: float, n_around: int) -> np.ndarray:
    """Closed-trailing-edge NACA 4-digit section, n_around points starting at the
    trailing edge, along the lower surface to the leading edge and back along the upper
    surface (clockwise around the body; half-cosine clustering)."""
    half = n_around // 2
    beta = np.linspace(0.0, math.pi, half + 1)
    # half cosine, half uniform: points gather towards the edges without making the
    # first triangle rings above the quad layers needle-shaped there
    xc = 0.25 * (1.0 - np.cos(beta)) + 0.5 * beta / math.pi  # 0 (LE) .. 1 (TE)
    yt = 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                    + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)
    if m > 0.0 and p > 0.0:
        yc = np.where(xc < p, m / p ** 2 * (2 * p * xc - xc ** 2),
                      m / (1 - p) ** 2 * ((1 - 2 * p) + 2 * p * xc - xc ** 2))
        dyc = np.where(xc < p, 2 * m / p ** 2 * (p - xc), 2 * m / (1 - p) ** 2 * (p - xc))
    else:
        yc = np.zeros_like(xc)
        dyc = np.zeros_like(xc)
    th = np.arctan(dyc)
    xu, yu = xc - yt * np.sin(th), yc + yt * np.cos(th)
    xl, yl = xc + yt * np.sin(th), yc - yt * np.cos(th)
    # TE -> lower surface -> LE -> upper surface
    lower = np.stack([xl[::-1], yl[::-1]], axis=1)      # TE .. LE
    upper = np.stack([xu[1:-1], yu[1:-1]], axis=1)      # after LE .. before TE
    pts = np.concatenate([lower, upper], axis=0)
    pts[0] = (1.0, 0.0)
    return pts[:n_around]


def _march_rings(inner: np.ndarray, h0: float, n_rings: int, r_far: float, centre: np.ndarray):
    """Rings of an O-grid from the closed curve `inner` (clockwise, fluid on the left of
    its tangent) out to the circle of radius r_far about `centre`: each ring steps from
    the previous one along its smoothed left normal, by steps growing geometrically from
    h0, and is then smoothed along itself (which rounds it and evens out its spacing);
    over the outer third the rings are blended onto circles, the last one onto the far
    circle. Marching normals of a rounding curve do not cross, so no cell folds."""
    n = inner.shape[0]
    d_far = r_far - np.linalg.norm(inner - centre, axis=1).mean()
    q = _solve_ratio(h0, d_far, n_rings)
    steps = h0 * q ** np.arange(n_rings)
    rings, X = [], inner.copy()
    k_blend = int(round(0.65 * n_rings))
    for k in range(n_rings):
        t = np.roll(X, -1, axis=0) - np.roll(X, 1, axis=0)
        nrm = np.stack([-t[:, 1], t[:, 0]], axis=1)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        for _ in range(2 + k // 4):
            nrm = nrm + 0.5 * (np.roll(nrm, 1, axis=0) + np.roll(nrm, -1, axis=0))
            nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        X = X + steps[k] * nrm
        nu = min(0.5, 0.05 + 0.45 * k / n_rings)
        for _ in range(2):
            X = X + nu * (0.5 * (np.roll(X, 1, axis=0) + np.roll(X, -1, axis=0)) - X)
        # move the points along the ring towards even arc-length spacing (fully even from
        # 60% of the rings out), keeping point 0 in place: far from the body the cells
        # then have the same aspect ratio all around
        w = min(1.0, (k + 1) / (0.6 * n_rings))
        seg = np.linalg.norm(np.roll(X, -1, axis=0) - X, axis=1)
        s_pts = np.concatenate([[0.0], np.cumsum(seg)])
        L = s_pts[-1]
        target = (1.0 - w) * s_pts[:-1] + w * L * np.arange(n) / n
        Xc = np.concatenate([X, X[:1]], axis=0)
        X = np.stack([np.interp(target, s_pts, Xc[:, 0]), np.interp(target, s_pts, Xc[:, 1])], axis=1)
        if k >= k_blend:
            rel = X - centre
            rad = np.linalg.norm(rel, axis=1, keepdims=True)
            r_k = r_far if k == n_rings - 1 else rad.mean()
            w = 1.0 if k == n_rings - 1 else (k - k_blend + 1) / (n_rings - k_blend)
            X = (1.0 - w) * X + w * (centre + r_k * rel / rad)
        rings.append(X.copy())
    return rings


def naca_omesh(m: float = 0.0, p: float = 0.0, t: float = 0.12, n_around: int = 320,
               n_quad: int = 48, first: float = 1e-6, ratio: float = 1.2,
               n_rings: int = 70, r_far: float = 20.0, jitter: float = 0.25,
               seed: int = 3, name: str = "naca_omesh") -> Mesh:
    """Hybrid O-mesh around a NACA 4-digit section: n_around x n_quad body-fitted quad
    layers (first spacing `first`, growth `ratio`), then n_rings rings marched out to a
    circle of radius r_far centred at (0.5, 0) (see _march_rings), the ring cells split
    into seeded-random triangles and interior ring points jittered by up to +-jitter of
    the local spacing."""
    rng = np.random.default_rng(seed)
    surf = naca4_surface(m, p, t, n_around)
    n = surf.shape[0]
    # the surface runs clockwise around the body (TE, lower surface, LE, upper surface),
    # so the fluid lies to the left of the centred tangent: left normal = into the fluid
    tang = np.roll(surf, -1, axis=0) - np.roll(surf, 1, axis=0)
    tang /= np.linalg.norm(tang, axis=1, keepdims=True)
    nrm = np.stack([-tang[:, 1], tang[:, 0]], axis=1)
    offs = geometric_levels(first, ratio, n_quad)
    # extrusion directions: the wall normal at the wall, turning with height towards a
    # smoothed normal, so that the fan around the sharp trailing edge spreads over many
    # cells of the upper layers instead of one
    smooth = nrm.copy()
    for _ in range(max(8, n // 4)):
        smooth = smooth + 0.5 * (np.roll(smooth, 1, axis=0) + np.roll(smooth, -1, axis=0))
        smooth /= np.linalg.norm(smooth, axis=1, keepdims=True)
    layers = [surf.copy()]
    for l in range(1, len(offs)):
        w = offs[l] / offs[-1]
        dvec = (1.0 - w) * nrm + w * smooth
        dvec /= np.linalg.norm(dvec, axis=1, keepdims=True)
        layers.append(layers[-1] + (offs[l] - offs[l - 1]) * dvec)
    inner = layers[-1]
    h_last = offs[-1] - offs[-2]
    rings = _march_rings(inner, h_last * ratio, n_rings, r_far, np.array([0.5, 0.0]))
    # jitter interior ring points (not the quad top, not the far circle)
    base = [r.copy() for r in rings]
    disp = []
    for k in range(len(rings) - 1):
        prev = inner if k == 0 else rings[k - 1]
        nxt = rings[k + 1]
        rad = np.minimum(np.linalg.norm(rings[k] - prev, axis=1),
                         np.linalg.norm(nxt - rings[k], axis=1))
        tangl = np.minimum(np.linalg.norm(rings[k] - np.roll(rings[k], 1, axis=0), axis=1),
                           np.linalg.norm(np.roll(rings[k], -1, axis=0) - rings[k], axis=1))
        lim = jitter * np.minimum(rad, tangl)
        disp.append(lim[:, None] * rng.uniform(-1.0, 1.0, size=(n, 2)) / math.sqrt(2.0))
    disp.append(np.zeros((n, 2)))
    nid = lambda i, l: l * n + (i % n)
    cells = []
    for l in range(n_quad):
        for i in range(n):
            # i -> i+1 along layer l has layer l+1 on its left: CCW cell
            cells.append([nid(i, l), nid(i + 1, l), nid(i + 1, l + 1), nid(i, l + 1)])
    diag = rng.integers(0, 2, size=(n_rings, n))
    tri = []
    for k in range(n_rings):
        l = n_quad + k
        for i in range(n):
            a, b, c, d = nid(i, l), nid(i + 1, l), nid(i + 1, l + 1), nid(i, l + 1)
            if diag[k, i] == 0:
                tri.append([a, b, c]); tri.append([a, c, d])
            else:
                tri.append([a, b, d]); tri.append([b, c, d])
    tri = np.asarray(tri)
    cells.extend(tri.tolist())
    # thin cells near a sharp trailing edge: undo the jitter of the nodes of any triangle
    # it inverted, and split a ring quad along its other diagonal when the chosen one
    # inverts, until every triangle is counter-clockwise
    n_fixed = (n_quad + 1) * n

    def tri_area(xy, t):
        P = xy[t]
        return 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                      - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    for _ in range(20):
        xy = np.concatenate(layers + [b_ + d_ for b_, d_ in zip(base, disp)], axis=0)
        area = tri_area(xy, tri)
        if np.all(area > 0.0):
            break
        for q in np.unique(np.nonzero(area <= 0.0)[0] // 2):
            k, i = divmod(q, n)
            l = n_quad + k
            a, b, c, d = nid(i, l), nid(i + 1, l), nid(i + 1, l + 1), nid(i, l + 1)
            alt = np.array([[a, b, d], [b, c, d]]) if diag[k, i] == 0 else np.array([[a, b, c], [a, c, d]])
            if np.all(tri_area(xy, alt) > 0.0):
                diag[k, i] = 1 - diag[k, i]
                tri[2 * q:2 * q + 2] = alt
            else:
                for g in {a, b, c, d}:
                    if g >= n_fixed:
                        disp[(g - n_fixed) // n][(g - n_fixed) % n] = 0.0
    cells = cells[:n_quad * n] + tri.tolist()
    wall_nodes = n  # nodes 0..n-1 are on the body

    def bc(a, b, xm, ym):
        if a < wall_nodes and b < wall_nodes:
            return BC_WALL
        return BC_FARFIELD
    mesh = build_mesh(xy, cells, bc, name=name)
    mesh.meta = dict(kind="naca", m=m, p=p, t=t, n_around=n_around, n_quad=n_quad,
                     n_rings=n_rings, first=first, ratio=ratio, seed=seed)
    return mesh


# --------------------------------------------------------------------------------------
# small meshes for unit checks
# --------------------------------------------------------------------------------------

def tiny_quads(nx: int = 2, ny: int = 2, skew: float = 0.0, seed: int = 0,
               bcs=("wall", "farfield")) -> Mesh:
    """nx x ny quads on [0,1]^2 (optionally with jittered interior nodes). Bottom edge
    is wall (or symmetry), the rest free stream (or as bcs[1] says)."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    X = X.copy(); Y = Y.copy()
    if skew > 0:
        for j in range(1, ny):
            for i in range(1, nx):
                X[j, i] += skew / nx * rng.uniform(-1, 1)
                Y[j, i] += skew / ny * rng.uniform(-1, 1)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    nid = lambda i, j: j * (nx + 1) + i
    cells = [[nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)]
             for j in range(ny) for i in range(nx)]
    tags = {"wall": BC_WALL, "symmetry": BC_SYMMETRY, "farfield": BC_FARFIELD, "outflow": BC_OUTFLOW}
    bottom, other = tags[bcs[0]], tags[bcs[1]]
    return build_mesh(xy, cells, lambda a, b, xm, ym: bottom if abs(ym) < 1e-12 else other,
                      name=f"tiny_quads_{nx}x{ny}")


def triangle_fan(n: int = 4, radius: float = 1.0) -> Mesh:
    """n triangles around a centre node; the outer edges are free stream."""
    ang = np.linspace(0.0, 2 * math.pi, n, endpoint=False) + 0.3
    xy = np.concatenate([[[0.0, 0.0]], np.stack([radius * np.cos(ang), radius * np.sin(ang)], 1)])
    cells = [[0, 1 + k, 1 + (k + 1) % n] for k in range(n)]
    return build_mesh(xy, cells, lambda a, b, xm, ym: BC_FARFIELD, name=f"fan{n}")


def mixed_polygons(seed: int = 0) -> Mesh:
    """A small mesh of eight cells: six quads, one pentagon and one triangle (general
    polygons as in the paper's hybrid meshes). Bottom is wall, the right side outflow, the
    rest free stream."""
    xy = np.array([
        [0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [3.0, 0.0],      # 0..3 bottom
        [0.0, 1.0], [1.0, 1.0], [2.0, 1.0], [3.0, 1.0],      # 4..7
        [1.5, 1.2],                                           # 8 (pentagon apex)
        [0.0, 2.0], [1.0, 2.2], [2.0, 2.2], [3.0, 2.0],      # 9..12
        [2.5, 1.6],                                           # 13 (hexagon side)
    ], dtype=np.float64)
    cells = [
        [0, 1, 5, 4],            # quad
        [1, 2, 6, 8, 5],         # pentagon
        [2, 3, 7, 6],            # quad
        [4, 5, 10, 9],           # quad
        [5, 8, 11, 10],          # quad
        [6, 7, 12, 13],          # quad
        [8, 6, 13, 11],          # quad
        [13, 12, 11],            # triangle
    ]
    return build_mesh(xy, cells, lambda a, b, xm, ym: BC_WALL if abs(ym) < 1e-12 else
                      (BC_OUTFLOW if abs(xm - 3.0) < 1e-12 else BC_FARFIELD), name="mixed_polygons")


# --------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------

def laminar_plate() -> Mesh:
    """Laminar flat plate: 64 x 32 quads, y ratio 1.1 (2048 cells)."""
    return flat_plate_quads(64, 32, 1.1, name="laminar_plate_64x32")


def turbulent_plate(seed: int = 1) -> Mesh:
    """Turbulent flat plate: 128 x 64 quad layer + 128 x 48 x 2 triangles (20480 cells)."""
    return flat_plate_hybrid(seed=seed, name="turbulent_plate_20480")


def naca0012(seed: int = 3) -> Mesh:
    """NACA 0012 hybrid O-mesh, 320 x 48 quads + 320 x 70 x 2 triangles (60160 cells)."""
    return naca_omesh(0.0, 0.0, 0.12, seed=seed, name="naca0012_60160")


def naca_scaled(m: float, p: float, t: float, target_cells: int, seed: int, name: str = "") -> Mesh:
    """A NACA 4-digit O-mesh built like the NACA 0012 workload with its point and layer
    counts scaled by sqrt(target_cells / 60160) (cells = n_around (n_quad + 2 n_rings))."""
    s = math.sqrt(target_cells / 60160.0)
    n_around = max(64, 2 * int(round(160 * s)))
    n_quad = max(12, int(round(48 * s)))
    n_rings = max(8, int(round(70 * s)))
    # keep the quad layer as thick as the full-size one (first spacing 1e-6, 48 layers,
    # ratio 1.2): the growth ratio follows from the layer count
    height = geometric_levels(1e-6, 1.2, 48)[-1]
    ratio = _solve_ratio(1e-6, height, n_quad)
    return naca_omesh(m, p, t, n_around=n_around, n_quad=n_quad, ratio=ratio, n_rings=n_rings, seed=seed,
                      name=name or f"naca{m:.3f}_{p:.2f}_{t:.2f}_{n_around}x{n_quad}+{n_rings}")


def plate_scaled(target_cells: int, seed: int, name: str = "") -> Mesh:
    """A hybrid flat plate built like the 20480-cell turbulent plate with its point and
    layer counts scaled by sqrt(target_cells / 20480) (cells = nx (nq + 2 ntri_rows)),
    keeping the quad layer as thick as the full-size one (first spacing 1e-6)."""
    s = math.sqrt(target_cells / 20480.0)
    nx = max(16, int(round(128 * s)))
    nq = max(8, int(round(64 * s)))
    ntri = max(4, int(round(48 * s)))
    height = geometric_levels(1e-6, 1.15, 64)[-1]
    ratio = _solve_ratio(1e-6, height, nq)
    return flat_plate_hybrid(nx=nx, nq=nq, ntri_rows=ntri, first=1e-6, ratio=ratio, seed=seed,
                             name=name or f"plate_{nx}x{nq}+{ntri}")


def naca_batch_specs(n: int = 64, seed: int = 4, cells_lo: int = 8000, cells_hi: int = 80000):
    """Seeded parameters of the batched-airfoil workload: per case the NACA 4-digit shape
    (m in [0, 0.06], p in [0.2, 0.6], t in [0.08, 0.18]), the flow (Ma in [0.1, 0.75],
    AoA in [-4, 8] deg, Re_c log-uniform in [1e6, 1e7]) and a target cell count drawn
    log-uniform in [cells_lo, cells_hi]. Case i uses seed 1000 * seed + i for its mesh."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        specs.append(dict(
            m=float(rng.uniform(0.0, 0.06)), p=float(rng.uniform(0.2, 0.6)), t=float(rng.uniform(0.08, 0.18)),
            mach=float(rng.uniform(0.1, 0.75)), aoa=float(rng.uniform(-4.0, 8.0)),
            reynolds=float(10 ** rng.uniform(6.0, 7.0)),
            cells=int(round(10 ** rng.uniform(math.log10(cells_lo), math.log10(cells_hi)))),
            mesh_seed=1000 * seed + i))
    return specs


def serving_specs(n: int = 200, seed: int = 5, cells_lo: int = 2000, cells_hi: int = 250000):
    """Seeded request stream of the serving workload: per request a case (flat plate or
    NACA 4-digit section, probability 1/2 each), a target cell count log-uniform in
    [cells_lo, cells_hi], the flow (Ma in [0.1, 0.75], AoA in [-4, 8] deg for sections and
    0 for plates, Re log-uniform in [1e6, 1e7]), the section shape (m in [0, 0.06], p in
    [0.2, 0.6], t in [0.08, 0.18]) and an exponential inter-arrival gap of mean 1 (the
    caller scales it to the arrival rate). Request i uses seed 1000 * seed + i for its mesh."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(dict(
            kind="plate" if rng.uniform() < 0.5 else "naca",
            cells=int(round(10 ** rng.uniform(math.log10(cells_lo), math.log10(cells_hi)))),
            mach=float(rng.uniform(0.1, 0.75)), aoa=float(rng.uniform(-4.0, 8.0)),
            reynolds=float(10 ** rng.uniform(6.0, 7.0)),
            m=float(rng.uniform(0.0, 0.06)), p=float(rng.uniform(0.2, 0.6)), t=float(rng.uniform(0.08, 0.18)),
            gap=float(rng.exponential(1.0)), mesh_seed=1000 * seed + i))
    return out


def cavity(n: int = 100) -> Mesh:
    """Lid-driven cavity: n x n uniform quads on the unit square, fixed non-slip walls on
    the bottom and sides, the top a wall moving with the free-stream velocity (the lid)."""
    xs = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    nid = lambda i, j: j * (n + 1) + i
    cells = [[nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)] for j in range(n) for i in range(n)]
    m = build_mesh(xy, cells, lambda a, b, xm, ym: BC_MOVING_WALL if abs(ym - 1.0) < 1e-12 else BC_WALL,
                   name=f"cavity_{n}x{n}")
    m.meta = dict(kind="cavity", n=n)
    return m


def refined_cavity(n: int = 24, band: int = 3, patch=(0.5, 0.6, 0.16), jitter: float = 0.05,
                   seed: int = 0, permute_seed=None) -> Mesh:
    """Lid-driven cavity on an adaptively refined mesh of the kind the paper's second cavity
    mesh is (quads, pentagons and hexagons): an n x n coarse grid on the unit square whose
    cells within `band` cells of a wall, or with their centre inside the disc `patch`
    (x, y, radius), are split into 2 x 2 quads. A coarse cell next to refined ones keeps
    the refined side's middle node (a hanging node), so it becomes a pentagon (one refined
    neighbour), a hexagon (two) or a polygon of up to eight nodes. Interior nodes are moved
    by a seeded `jitter` x the fine spacing so that the polygons are not degenerate.
    Cells are numbered by centroid (rows from the bottom), or by a seeded random
    permutation (`permute_seed`), which gives cells with five or more lower or upper
    neighbours in the LU-SGS sweep order. Walls as in `cavity`."""
    rng = np.random.default_rng(seed)
    m2 = 2 * n + 1
    px, py, pr = patch
    h = 1.0 / n
    ref = np.zeros((n, n), dtype=bool)
    for j in range(n):
        for i in range(n):
            near = min(i, j, n - 1 - i, n - 1 - j) < band
            xc, yc = (i + 0.5) * h, (j + 0.5) * h
            ref[j, i] = near or (xc - px) ** 2 + (yc - py) ** 2 <= pr * pr
    lid = lambda I, J: J * m2 + I
    cells = []
    for j in range(n):
        for i in range(n):
            I, J = 2 * i, 2 * j
            if ref[j, i]:
                for b in range(2):
                    for a in range(2):
                        cells.append([lid(I + a, J + b), lid(I + a + 1, J + b), lid(I + a + 1, J + b + 1),
                                      lid(I + a, J + b + 1)])
                continue
            refined = lambda ii, jj: 0 <= ii < n and 0 <= jj < n and ref[jj, ii]
            poly = [lid(I, J)]
            if refined(i, j - 1):
                poly.append(lid(I + 1, J))
            poly.append(lid(I + 2, J))
            if refined(i + 1, j):
                poly.append(lid(I + 2, J + 1))
            poly.append(lid(I + 2, J + 2))
            if refined(i, j + 1):
                poly.append(lid(I + 1, J + 2))
            poly.append(lid(I, J + 2))
            if refined(i - 1, j):
                poly.append(lid(I, J + 1))
            cells.append(poly)
    used = np.unique(np.concatenate([np.asarray(c) for c in cells]))
    remap = -np.ones(m2 * m2, dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    I, J = used % m2, used // m2
    xy = np.stack([I / (2.0 * n), J / (2.0 * n)], axis=1)
    inner = (I > 0) & (I < 2 * n) & (J > 0) & (J < 2 * n)
    xy[inner] += jitter * (0.5 * h) * rng.uniform(-1.0, 1.0, size=(int(inner.sum()), 2))
    cells = [[int(remap[v]) for v in c] for c in cells]
    cen = np.array([xy[c].mean(axis=0) for c in cells])
    if permute_seed is None:
        order = np.lexsort((cen[:, 0], np.round(cen[:, 1], 9)))
    else:
        order = np.random.default_rng(permute_seed).permutation(len(cells))
    cells = [cells[k] for k in order]
    mesh = build_mesh(xy, cells, lambda a, b, xm, ym: BC_MOVING_WALL if abs(ym - 1.0) < 1e-12 else BC_WALL,
                      name=f"refined_cavity_{n}")
    mesh.meta = dict(kind="refined_cavity", n=n)
    return mesh
