"""Seeded triangle-soup generators (float32 [ntri, 3, 3], grid units: cell (i,j,k) spans [i,i+1)x[j,j+1)x[k,k+1)).

The shapes follow the paper's test geometries in kind only (Sec. 3.3 dirty sphere, Sec. 3.2 flat
plate, Sec. 3.1 bluff body, Sec. 3.4 vehicle-like assemblies); the paper's own CAD files are not
available, so every soup here is synthetic and reproducible from its seed.  A soup carries no
connectivity: triangles are independent, may overlap, leave gaps or be nested (Sec. 2.4, issues 1-5).
"""
import numpy as np

F32 = np.float32


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(subdiv, radius, center, dtype=F32):
    """Closed icosphere with 20*4**subdiv outward-oriented triangles."""
    v, f = _icosahedron()
    for _ in range(subdiv):
        edge_mid = {}
        verts = list(v)
        nf = []
        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in edge_mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                edge_mid[key] = len(verts) - 1
            return edge_mid[key]
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        v = np.array(verts)
        f = np.array(nf, dtype=np.int64)
    tri = v[f] * radius + np.asarray(center, dtype=np.float64)
    return tri.astype(dtype)


def _quad_grid(p0, eu, ev, m, n):
    """Tessellate the parallelogram p0 + s*eu + t*ev, s,t in [0,1], into m x n quads (2 triangles each)."""
    s = np.linspace(0.0, 1.0, m + 1)
    t = np.linspace(0.0, 1.0, n + 1)
    S, T = np.meshgrid(s, t, indexing="ij")
    P = p0[None, None, :] + S[..., None] * eu[None, None, :] + T[..., None] * ev[None, None, :]
    a = P[:-1, :-1].reshape(-1, 3)
    b = P[1:, :-1].reshape(-1, 3)
    c = P[1:, 1:].reshape(-1, 3)
    d = P[:-1, 1:].reshape(-1, 3)
    return np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)


def axis_box(lo, hi, m=1, dtype=F32):
    """Closed axis-aligned box [lo, hi], each face split into m x m quads (12*m*m triangles)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    e = hi - lo
    ex, ey, ez = np.diag(e)
    faces = [
        _quad_grid(lo, ey, ez, m, m),                    # x = lo
        _quad_grid(lo + ex, ez, ey, m, m),               # x = hi
        _quad_grid(lo, ez, ex, m, m),                    # y = lo
        _quad_grid(lo + ey, ex, ez, m, m),               # y = hi
        _quad_grid(lo, ex, ey, m, m),                    # z = lo
        _quad_grid(lo + ez, ey, ex, m, m),               # z = hi
    ]
    return np.concatenate(faces, 0).astype(dtype)


def fan_disk(center, radius, normal_axis, nseg, dtype=F32):
    """Zero-thickness disk as an nseg-triangle fan around its centre."""
    c = np.asarray(center, np.float64)
    a = normal_axis
    b, d = (a + 1) % 3, (a + 2) % 3
    th = np.linspace(0.0, 2.0 * np.pi, nseg + 1)
    rim = np.zeros((nseg + 1, 3))
    rim[:, b] = radius * np.cos(th)
    rim[:, d] = radius * np.sin(th)
    rim += c
    tri = np.stack([np.broadcast_to(c, (nseg, 3)), rim[:-1], rim[1:]], 1)
    return tri.astype(dtype)


def _cylinder(center, radius, length, axis, nseg, nlen):
    c = np.asarray(center, np.float64)
    b, d = (axis + 1) % 3, (axis + 2) % 3
    th = np.linspace(0.0, 2.0 * np.pi, nseg + 1)
    z = np.linspace(-0.5 * length, 0.5 * length, nlen + 1)
    TH, Z = np.meshgrid(th, z, indexing="ij")
    P = np.zeros(TH.shape + (3,))
    P[..., b] = radius * np.cos(TH)
    P[..., d] = radius * np.sin(TH)
    P[..., axis] = Z
    P += c
    a_ = P[:-1, :-1].reshape(-1, 3)
    b_ = P[1:, :-1].reshape(-1, 3)
    c_ = P[1:, 1:].reshape(-1, 3)
    d_ = P[:-1, 1:].reshape(-1, 3)
    side = np.concatenate([np.stack([a_, b_, c_], 1), np.stack([a_, c_, d_], 1)], 0)
    caps = []
    for zc in (-0.5 * length, 0.5 * length):
        cc = c.copy()
        cc[axis] += zc
        disk = fan_disk(cc, radius, axis, nseg, dtype=np.float64)
        caps.append(disk)
    return np.concatenate([side] + caps, 0)


def prism_2d(polygon, z_lo, z_hi, dtype=F32):
    """Open lateral surface of a prism along z over a closed polygon [(x, y), ...] (first point
    repeated at the end): two triangles per edge, no caps.  Extending it past both z faces of a grid
    gives a 2-D body for quasi-two-dimensional runs."""
    P = np.asarray(polygon, np.float64)
    tri = []
    for a, b in zip(P[:-1], P[1:]):
        A0, B0 = [a[0], a[1], z_lo], [b[0], b[1], z_lo]
        A1, B1 = [a[0], a[1], z_hi], [b[0], b[1], z_hi]
        tri.append([A0, B0, B1])
        tri.append([A0, B1, A1])
    return np.array(tri).astype(dtype)


def taylor_green_body(n, nz, shape="circle", lo=-2.0, hi=2.0, nseg=256):
    """The immersed bodies of the Taylor-Green verification (Sec. 2.5) in grid units of an n x n x nz
    grid on [lo, hi]^2: a circle of radius 1 ("circle", nseg edges) or the square of side sqrt(2)
    inscribed in it, turned 45 degrees ("diamond", corners on the axes, 8 edges per side), both
    centred at the origin and extended 3 cells past the z faces."""
    dx = (hi - lo) / n
    c = np.array([-lo / dx, -lo / dx])
    r = 1.0 / dx
    if shape == "circle":
        th = np.linspace(0.0, 2.0 * np.pi, nseg + 1)
        poly = c + r * np.stack([np.cos(th), np.sin(th)], 1)
    elif shape == "diamond":
        corners = np.array([[r, 0.0], [0.0, r], [-r, 0.0], [0.0, -r], [r, 0.0]])
        s = np.linspace(0.0, 1.0, 9)[:-1]
        poly = np.concatenate([a + s[:, None] * (b - a) for a, b in zip(corners[:-1], corners[1:])]
                              + [corners[-1:]]) + c
    else:
        raise ValueError(shape)
    return prism_2d(poly, -3.0, nz + 3.0)


def _rot_y(tri, angle_deg, pivot):
    a = np.deg2rad(angle_deg)
    R = np.array([[np.cos(a), 0.0, np.sin(a)], [0.0, 1.0, 0.0], [-np.sin(a), 0.0, np.cos(a)]])
    p = np.asarray(pivot, np.float64)
    return (tri - p) @ R.T + p


def dirty_sphere(seed=2, radius=16.0, center=(64.0, 64.0, 64.0), subdiv=5,
                 dup_frac=0.02, del_frac=0.05, jitter=0.02, inner_ratio=0.7, disk_ratio=0.6,
                 disk_seg=256):
    """Dirty sphere of Sec. 3.3 (synthetic stand-in): duplicates offset 0.1 along the normal
    (overlaps), deleted faces (holes), vertex jitter (cracks), a nested inner shell and a
    zero-thickness disk through the centre."""
    rng = np.random.default_rng(seed)
    tri = icosphere(subdiv, radius, center, dtype=np.float64)
    n = len(tri)
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dup = rng.choice(n, size=int(round(dup_frac * n)), replace=False)
    tri = np.concatenate([tri, tri[dup] + 0.1 * nrm[dup][:, None, :]], 0)
    keep = np.ones(len(tri), bool)
    keep[rng.choice(len(tri), size=int(round(del_frac * n)), replace=False)] = False
    tri = tri[keep]
    tri = tri + rng.normal(0.0, jitter, size=tri.shape)
    inner = icosphere(subdiv, inner_ratio * 2 * radius / 2.0, center, dtype=np.float64)
    disk = fan_disk(center, disk_ratio * 2 * radius / 2.0, 0, disk_seg, dtype=np.float64)
    return np.concatenate([tri, inner, disk], 0).astype(F32)


def cube_and_plate():
    """Bluff body on the floor plus an inclined zero-thickness plate (Sec. 3.1/3.2 stand-in).

    Cube [112,144]x[112,144]x[0,32], two triangles per face, adjacent faces shifted by 1e-3 so the
    edges leave cracks, one face re-split into 2+4 triangles (T-junctions).  Plate 64x64 at 10 deg
    incidence about y, centred at (256,128,64), 2 triangles plus a 4-triangle half (T-junctions)."""
    lo = np.array([112.0, 112.0, 0.0])
    hi = np.array([144.0, 144.0, 32.0])
    faces = []
    box = axis_box(lo, hi, 1, dtype=np.float64).reshape(6, 2, 3, 3)
    for fi in range(6):
        shift = np.zeros(3)
        shift[fi // 2] = (1e-3 if fi % 2 else -1e-3)
        f = box[fi] + shift
        if fi == 3:  # y = hi face: split into a 2-triangle half and a 4-triangle half
            p0 = np.array([lo[0], hi[1], lo[2]]) + shift
            ex = np.array([hi[0] - lo[0], 0, 0])
            ez = np.array([0, 0, hi[2] - lo[2]])
            f = np.concatenate([_quad_grid(p0, 0.5 * ex, ez, 1, 1),
                                _quad_grid(p0 + 0.5 * ex, 0.5 * ex, 0.5 * ez, 1, 2)], 0)
        faces.append(f)
    c = np.array([256.0, 128.0, 64.0])
    p0 = c - np.array([32.0, 32.0, 0.0])
    plate = np.concatenate([_quad_grid(p0, np.array([32.0, 0, 0]), np.array([0, 64.0, 0]), 1, 1),
                            _quad_grid(p0 + np.array([32.0, 0, 0]), np.array([32.0, 0, 0]),
                                       np.array([0, 32.0, 0]), 1, 2)], 0)
    plate = _rot_y(plate, 10.0, c)
    tri = np.concatenate(faces + [plate], 0)
    return tri.astype(F32)


def vehicle_assembly(seed=4, nparts=300, target_tris=2_000_000,
                     envelope_lo=(192.0, 136.0, 16.0), envelope_hi=(832.0, 376.0, 176.0)):
    """Vehicle-like dirty assembly (Sec. 3.4 stand-in): a union of boxes, cylinders and
    zero-thickness plates that overlap, interpenetrate, nest and leave gaps of up to 0.5 cells."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(envelope_lo)
    hi = np.asarray(envelope_hi)
    ext = hi - lo
    per_part = target_tris / nparts
    parts = []
    # a main body block so that most parts touch or sit inside something
    body_lo = lo + np.array([0.0, 0.0, 20.0])
    body_hi = hi - np.array([0.0, 0.0, 40.0])
    m = max(1, int(round((per_part / 12) ** 0.5)))
    parts.append(axis_box(body_lo, body_hi, m, dtype=np.float64))
    prev_hi = None
    for p in range(1, nparts):
        kind = rng.integers(0, 3)
        size = rng.uniform(8.0, 120.0, size=3) * np.array([1.0, 0.6, 0.4])
        cen = lo + rng.uniform(0.0, 1.0, size=3) * ext
        if prev_hi is not None and rng.uniform() < 0.3:
            # butt against the previous part with a small gap (<= 0.5 cells)
            cen = prev_hi + rng.uniform(0.0, 0.5) + 0.5 * size * np.array([1.0, 0.0, 0.0])
        cen = np.clip(cen, lo + 0.5 * size, hi - 0.5 * size)
        if kind == 0:
            mm = max(1, int(round((per_part / 12) ** 0.5)))
            t = axis_box(cen - 0.5 * size, cen + 0.5 * size, mm, dtype=np.float64)
        elif kind == 1:
            nseg = int(rng.integers(32, 97))
            nlen = max(1, int(round((per_part - 2 * nseg) / (2 * nseg))))
            axis = int(rng.integers(0, 3))
            t = _cylinder(cen, 0.5 * min(size[(axis + 1) % 3], size[(axis + 2) % 3]),
                          size[axis], axis, nseg, nlen)
        else:
            mm = max(1, int(round((per_part / 2) ** 0.5)))
            axis = int(rng.integers(0, 3))
            b, d = (axis + 1) % 3, (axis + 2) % 3
            eu = np.zeros(3); eu[b] = size[b]
            ev = np.zeros(3); ev[d] = size[d]
            t = _quad_grid(cen - 0.5 * eu - 0.5 * ev, eu, ev, mm, mm)
            t = _rot_y(t, rng.uniform(-20.0, 20.0), cen)
        prev_hi = cen + 0.5 * size
        parts.append(t)
    return np.concatenate(parts, 0).astype(F32)


def random_soup(ntri, lo, hi, size, seed):
    """Independent random triangles inside [lo, hi] with edge lengths up to `size` (for predicate tests)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    a = lo + rng.uniform(0.0, 1.0, size=(ntri, 3)) * (hi - lo)
    b = a + rng.uniform(-size, size, size=(ntri, 3))
    c = a + rng.uniform(-size, size, size=(ntri, 3))
    return np.stack([a, b, c], 1).astype(F32)
