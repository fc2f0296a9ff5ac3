"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates inputs (geometry, receivers, frequencies); it holds
none of the field method's arithmetic.  Both the CUDA library's callers and
the FP64 oracle read the arrays it returns, so every coordinate is rounded to
float32 once here and both sides see identical values.

Workloads (the paper's Sec. III.C / IV describe rooms with PEC balls and a
PEC-cylinder stand-in for people; its scenes are not published, so these
stand in for them):
  * ``sphere_ring``  -- PEC sphere a = 0.5 m at the origin, source at (3, 0, 0),
    4096 receivers on the radius-2 m ring in z = 0, 2.4 GHz (Sec. IV.A's
    analytical-sphere validation, at a fixed size).
  * ``room``         -- 10 x 8 x 3 m box (6 PEC faces as 12 triangles) with N
    PEC cylinders (radius U[0.15, 0.25] m, height 1.7 m, on the floor),
    source at (1, 1, 2), receiver grid at z = 1.2 m.
  * ``crowd``        -- frames of that room in which the cylinders (people)
    walk: every 0.1 s each takes a 0.14 m step (1.4 m/s) in a random
    direction, kept inside the room, clear of the source and of each other
    (Sec. III's dynamic scenes); per frame its own frequencies (uniform in a
    band) and an uneven receiver count (log-uniform), receivers uniform over
    the floor plan at z = 1.2 m.
"""
import numpy as np

C0 = 299792458.0
SEED_BASE = 2310101

BODY_SPHERE = 0
BODY_CYLINDER = 1


class Scene:
    """Plain container: float32 arrays, no behaviour."""

    def __init__(self, tri, tri_face, bodies, tx, pol, freqs, rx, name, max_order=2, face_eps=None):
        self.tri = np.ascontiguousarray(tri, dtype=np.float32).reshape(-1, 3, 3)
        self.tri_face = np.ascontiguousarray(tri_face, dtype=np.int32)
        self.bodies = np.ascontiguousarray(bodies, dtype=np.float32).reshape(-1, 6)
        self.tx = np.asarray(tx, dtype=np.float32).reshape(3)
        self.pol = np.asarray(pol, dtype=np.float32).reshape(3)
        self.freqs = np.asarray(freqs, dtype=np.float64).reshape(-1)
        self.rx = np.ascontiguousarray(rx, dtype=np.float32).reshape(-1, 3)
        self.name = name
        self.max_order = int(max_order)
        # per face (dielectric flag, eps', eps''), eps_r = eps' - j eps''; None: every face PEC
        self.face_eps = None if face_eps is None else np.asarray(face_eps, dtype=np.float32).reshape(-1, 3)
        self.max_enc = 0          # extra encirclements of the creeping rays
        self.wall_creep = False   # creeping rays fed by one planar reflection
        self.candidates = None    # candidate face sequences [n, 3] of the planar paths (large scenes)

    @property
    def n_rx(self):
        return self.rx.shape[0]

    def rx_soa(self):
        """Receivers as a [3][n_rx] float32 array (x row, y row, z row)."""
        return np.ascontiguousarray(self.rx.T)

    def subset(self, idx, name=None):
        sub = Scene(self.tri, self.tri_face, self.bodies, self.tx, self.pol, self.freqs,
                    self.rx[idx], name or self.name + "[sub]", self.max_order, self.face_eps)
        sub.max_enc = self.max_enc
        sub.wall_creep = self.wall_creep
        sub.candidates = self.candidates
        return sub


def box_triangles(lx, ly, lz):
    """Axis-aligned box [0,lx]x[0,ly]x[0,lz] as 12 triangles, 2 per face.
    Face ids: 0 floor, 1 ceiling, 2 x=0, 3 x=lx, 4 y=0, 5 y=ly."""
    quads = [
        [(0, 0, 0), (lx, 0, 0), (lx, ly, 0), (0, ly, 0)],
        [(0, 0, lz), (0, ly, lz), (lx, ly, lz), (lx, 0, lz)],
        [(0, 0, 0), (0, ly, 0), (0, ly, lz), (0, 0, lz)],
        [(lx, 0, 0), (lx, 0, lz), (lx, ly, lz), (lx, ly, 0)],
        [(0, 0, 0), (0, 0, lz), (lx, 0, lz), (lx, 0, 0)],
        [(0, ly, 0), (lx, ly, 0), (lx, ly, lz), (0, ly, lz)],
    ]
    tri, face = [], []
    for f, q in enumerate(quads):
        tri.append([q[0], q[1], q[2]]); face.append(f)
        tri.append([q[0], q[2], q[3]]); face.append(f)
    return np.asarray(tri, dtype=np.float32), np.asarray(face, dtype=np.int32)


def sphere_ring(n_rx=4096, pol=(0.0, 0.0, 1.0), freq=2.4e9, radius=0.5, tx=(3.0, 0.0, 0.0), ring=2.0):
    phi = 2.0 * np.pi * np.arange(n_rx) / n_rx
    rx = np.stack([ring * np.cos(phi), ring * np.sin(phi), np.zeros(n_rx)], axis=1)
    bodies = np.array([[BODY_SPHERE, 0.0, 0.0, 0.0, radius, 0.0]])
    name = "sphere_ring(a=%.2f m, %d rx, pol=%s, %.2f GHz)" % (radius, n_rx, tuple(pol), freq / 1e9)
    return Scene(np.zeros((0, 3, 3)), np.zeros(0), bodies, tx, pol, [freq], rx, name, max_order=0)


def place_cylinders(n, lx, ly, rng, r_lo=0.15, r_hi=0.25, height=1.7, gap=0.05, avoid=None, max_tries=100000):
    """Non-overlapping vertical cylinders on the floor (>= gap between surfaces
    and >= gap from the walls).  ``avoid``: list of (x, y, clearance) points to
    keep outside every footprint."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d cylinders" % n)
        r = np.float32(rng.uniform(r_lo, r_hi))
        x = np.float32(rng.uniform(r + gap, lx - r - gap))
        y = np.float32(rng.uniform(r + gap, ly - r - gap))
        ok = True
        for (cx, cy, cr) in out:
            if np.hypot(x - cx, y - cy) < r + cr + gap:
                ok = False
                break
        if ok and avoid:
            for (px, py, cl) in avoid:
                if np.hypot(x - px, y - py) < r + cl:
                    ok = False
                    break
        if ok:
            out.append((x, y, r))
    return np.array([[BODY_CYLINDER, x, y, 0.0, r, height] for (x, y, r) in out], dtype=np.float32)


def grid_receivers(nx, ny, lx, ly, z):
    xs = (np.arange(nx) + 0.5) * (lx / nx)
    ys = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(xs, ys)          # row-major: y outer, x inner
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)


def room(n_cyl=20, nx=256, ny=256, freqs=(2.4e9, 5.8e9, 28e9), seed=SEED_BASE + 1,
         size=(10.0, 8.0, 3.0), tx=(1.0, 1.0, 2.0), pol=(0.0, 0.0, 1.0), rx_z=1.2, max_order=2, face_eps=None):
    """face_eps: None (PEC faces) or, per face id (floor, ceiling, x=0, x=lx,
    y=0, y=ly), None for PEC or (eps', eps'') of a dielectric half-space."""
    lx, ly, lz = size
    rng = np.random.default_rng(seed)
    tri, face = box_triangles(lx, ly, lz)
    bodies = place_cylinders(n_cyl, lx, ly, rng, avoid=[(tx[0], tx[1], 0.3)])
    rx = grid_receivers(nx, ny, lx, ly, rx_z)
    name = "room(%gx%gx%g m, %d PEC cylinders, %dx%d rx, f=%s GHz, refl<=%d%s)" % (
        lx, ly, lz, n_cyl, nx, ny, ",".join("%g" % (f / 1e9) for f in freqs), max_order,
        "" if face_eps is None else ", dielectric faces")
    fe = None
    if face_eps is not None:
        fe = [(0.0, 0.0, 0.0) if e is None else (1.0, float(e[0]), float(e[1])) for e in face_eps]
    return Scene(tri, face, bodies, tx, pol, freqs, rx, name, max_order=max_order, face_eps=fe)


def box_mesh(x0, x1, y0, y1, z0, z1, face0):
    """An axis-aligned box as 12 triangles, 2 per side, face ids face0 ..
    face0 + 5 (bottom, top, x0, x1, y0, y1)."""
    quads = [
        [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0)],
        [(x0, y0, z1), (x0, y1, z1), (x1, y1, z1), (x1, y0, z1)],
        [(x0, y0, z0), (x0, y1, z0), (x0, y1, z1), (x0, y0, z1)],
        [(x1, y0, z0), (x1, y0, z1), (x1, y1, z1), (x1, y1, z0)],
        [(x0, y0, z0), (x0, y0, z1), (x1, y0, z1), (x1, y0, z0)],
        [(x0, y1, z0), (x1, y1, z0), (x1, y1, z1), (x0, y1, z1)],
    ]
    tri, face = [], []
    for f, q in enumerate(quads):
        tri.append([q[0], q[1], q[2]]); face.append(face0 + f)
        tri.append([q[0], q[2], q[3]]); face.append(face0 + f)
    return tri, face


def office(n_rooms=(20, 15), room=(5.0, 4.0), height=3.0, n_furn=15000, n_cyl=100, n_sph=10, n_tx=4,
           nx=1250, ny=800, freqs=(5.8e9,), seed=SEED_BASE + 5, wall=0.12, door=1.0, rx_z=1.2, max_order=3):
    """Large office: a building of n_rooms[0] x n_rooms[1] rooms of room[0] x
    room[1] m, as axis-aligned boxes -- the outer shell, interior wall panels
    (thickness `wall`, a door gap of `door` m in every wall between two
    rooms) and furniture boxes on the floor with sides and height uniform in
    0.3-2 m -- each box 12 triangles and 6 faces; n_cyl PEC cylinders
    (radius 0.15-0.25 m, 1.7 m high) and n_sph PEC spheres (radius 0.1-0.4
    m, centre 0.5-2 m high); n_tx transmitters at 2.5 m in distinct room
    centres (scene.txs; scene.tx is the first); receivers on an nx x ny grid
    at rx_z.  Default: about 195k triangles, 1M receivers, 5.8 GHz."""
    rng = np.random.default_rng(seed)
    nrx, nry = n_rooms
    lx, ly = nrx * room[0], nry * room[1]
    tri, face = box_mesh(0.0, lx, 0.0, ly, 0.0, height, 0)
    nf = 6

    def add(x0, x1, y0, y1, z0, z1):
        nonlocal nf
        t, f = box_mesh(x0, x1, y0, y1, z0, z1, nf)
        tri.extend(t); face.extend(f)
        nf += 6

    h = wall / 2
    for j in range(1, nry):                      # walls along x between room rows
        y = j * room[1]
        for i in range(nrx):
            xa, xb = i * room[0], (i + 1) * room[0]
            g = rng.uniform(xa + 0.5, xb - 0.5 - door)
            add(xa, g, y - h, y + h, 0.0, height)
            add(g + door, xb, y - h, y + h, 0.0, height)
    for i in range(1, nrx):                      # walls along y between room columns
        x = i * room[0]
        for j in range(nry):
            ya, yb = j * room[1], (j + 1) * room[1]
            g = rng.uniform(ya + 0.5, yb - 0.5 - door)
            add(x - h, x + h, ya, g, 0.0, height)
            add(x - h, x + h, g + door, yb, 0.0, height)
    rooms = rng.choice(nrx * nry, n_tx, replace=False)
    txs = [((r % nrx + 0.5) * room[0] + 0.0123, (r // nrx + 0.5) * room[1] + 0.0171, 2.5) for r in rooms]
    for _ in range(n_furn):
        sx, sy, sz = rng.uniform(0.3, 2.0, 3)
        x0 = rng.uniform(0.2, lx - 0.2 - sx)
        y0 = rng.uniform(0.2, ly - 0.2 - sy)
        add(x0, x0 + sx, y0, y0 + sy, 0.0, sz)
    tri = np.asarray(tri, dtype=np.float32)
    face = np.asarray(face, dtype=np.int32)
    cyl = place_cylinders(n_cyl, lx, ly, rng, avoid=[(t[0], t[1], 0.3) for t in txs], max_tries=1000000)
    sph = []
    while len(sph) < n_sph:
        a = rng.uniform(0.1, 0.4)
        c = np.array([rng.uniform(a + 0.1, lx - a - 0.1), rng.uniform(a + 0.1, ly - a - 0.1), rng.uniform(0.5, 2.0)])
        if any(np.linalg.norm(c - np.asarray(t)) < a + 0.3 for t in txs):
            continue
        if any(np.hypot(*(c[:2] - b[1:3])) < a + b[4] + 0.05 for b in cyl):
            continue
        if any(np.linalg.norm(c - s_[1:4]) < a + s_[4] + 0.05 for s_ in sph):
            continue
        sph.append(np.array([BODY_SPHERE, *c, a, 0.0], dtype=np.float32))
    bodies = np.concatenate([cyl, np.asarray(sph, dtype=np.float32).reshape(-1, 6)], axis=0)
    rx = grid_receivers(nx, ny, lx, ly, rx_z)
    name = "office(%dx%d rooms, %d triangles, %d PEC cylinders + %d spheres, %dx%d rx, %d Tx, f=%s GHz, refl<=%d)" % (
        nrx, nry, tri.shape[0], n_cyl, n_sph, nx, ny, n_tx, ",".join("%g" % (f / 1e9) for f in freqs), max_order)
    sc = Scene(tri, face, bodies, txs[0], (0.0, 0.0, 1.0), freqs, rx, name, max_order=max_order)
    sc.txs = np.asarray(txs, dtype=np.float32)
    return sc


class Crowd:
    """Frames of one room: shared triangles, source and polarisation; per
    frame its bodies, frequencies and receivers (float32 arrays)."""

    def __init__(self, tri, tri_face, tx, pol, bodies, freqs, rx, name, max_order=2):
        self.tri, self.tri_face = tri, tri_face
        self.tx = np.asarray(tx, dtype=np.float32).reshape(3)
        self.pol = np.asarray(pol, dtype=np.float32).reshape(3)
        self.bodies = bodies          # list of [n_body, 6] float32
        self.freqs = freqs            # list of [n_f] float64
        self.rx = rx                  # list of [n_rx, 3] float32
        self.name = name
        self.max_order = int(max_order)

    @property
    def n_frames(self):
        return len(self.rx)

    @property
    def n_rx(self):
        return [r.shape[0] for r in self.rx]

    def frame(self, i, idx=None):
        """Frame i (or the receivers idx of it) as a single Scene."""
        rx = self.rx[i] if idx is None else self.rx[i][idx]
        return Scene(self.tri, self.tri_face, self.bodies[i], self.tx, self.pol, self.freqs[i], rx,
                     "%s[frame %d]" % (self.name, i), self.max_order)


def walk_step(bodies, lx, ly, rng, step, avoid, gap=0.05, tries=16):
    """One random-walk step of every cylinder (in order): a move of length
    `step` in a uniform random direction, redrawn up to `tries` times while
    it would leave the room (gap), overlap another cylinder (gap) or come
    within clearance of a point in `avoid`; a cylinder with no free move stays."""
    out = bodies.copy()
    for i in range(len(out)):
        r = float(out[i, 4])
        for _ in range(tries):
            th = rng.uniform(0.0, 2.0 * np.pi)
            x = np.float32(out[i, 1] + step * np.cos(th))
            y = np.float32(out[i, 2] + step * np.sin(th))
            if not (r + gap <= x <= lx - r - gap and r + gap <= y <= ly - r - gap):
                continue
            ok = True
            for j in range(len(out)):
                if j != i and np.hypot(x - out[j, 1], y - out[j, 2]) < r + out[j, 4] + gap:
                    ok = False
                    break
            if ok:
                for (px, py, cl) in avoid:
                    if np.hypot(x - px, y - py) < r + cl:
                        ok = False
                        break
            if ok:
                out[i, 1], out[i, 2] = x, y
                break
    return out


def crowd(n_frames=64, n_cyl=50, n_freq=16, band=(24e9, 30e9), rx_range=(1000, 65536), speed=1.4, dt=0.1,
          seed=SEED_BASE + 3, size=(10.0, 8.0, 3.0), tx=(1.0, 1.0, 2.0), pol=(0.0, 0.0, 1.0), rx_z=1.2,
          max_order=2):
    lx, ly, lz = size
    rng = np.random.default_rng(seed)
    tri, face = box_triangles(lx, ly, lz)
    avoid = [(tx[0], tx[1], 0.3)]
    b = place_cylinders(n_cyl, lx, ly, rng, avoid=avoid)
    bodies, freqs, rxs = [], [], []
    for f in range(n_frames):
        if f > 0:
            b = walk_step(b, lx, ly, rng, speed * dt, avoid)
        bodies.append(b.copy())
        freqs.append(rng.uniform(band[0], band[1], n_freq))
        n = int(round(np.exp(rng.uniform(np.log(rx_range[0]), np.log(rx_range[1])))))
        rx = np.stack([rng.uniform(0.0, lx, n), rng.uniform(0.0, ly, n), np.full(n, rx_z)], axis=1)
        rxs.append(np.ascontiguousarray(rx, dtype=np.float32))
    name = "crowd(%d frames, %gx%gx%g m, %d walking PEC cylinders, %d freqs in %g-%g GHz, rx %d-%d log-uniform)" % (
        n_frames, lx, ly, lz, n_cyl, n_freq, band[0] / 1e9, band[1] / 1e9, rx_range[0], rx_range[1])
    return Crowd(tri, face, tx, pol, bodies, freqs, rxs, name, max_order=max_order)
