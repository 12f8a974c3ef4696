"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws random numbers and builds input structure (decoder
weights, a regular tet grid, lumped masses, cubature sets, latent states).  It
holds none of the method's arithmetic: no decoder evaluation, no derivatives,
no forces.  Both the CUDA library and the FP64 oracle consume the arrays it
returns, so neither side depends on the other.

Workloads (the paper ships no meshes or trained decoders, so these stand in):

* ``small``  -- latent r=5, widths 5-64-256-1024-3000 (1000 vertices on a
  10x10x10 grid, 3645 tets), tanh, StVK E=1e5 nu=0.4, 64 cubature tets.
* ``paper``  -- latent r=30, ten layers 30-128-256-512-1024-2048-2048-2048-
  4096-4096-60000 (20x20x50 grid, 88445 tets), tanh, Neo-Hookean E=5e5
  nu=0.45, 500 cubature tets, gravity.  Decoder depth ("10+ layers", Sec. 1),
  latent size ("below a couple of dozens", Sec. 3.5) and cubature counts
  (Table 2: 100-11400) follow the paper's reported scale.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GRAVITY = 9.81


@dataclasses.dataclass
class Decoder:
    widths: list            # [r, n_1, ..., N]
    W: list                 # W[l]: float32 (n_out, n_in), row-major
    b: list                 # b[l]: float32 (n_out,)
    act: str = "tanh"       # hidden activation: tanh | sin | linear

    @property
    def r(self):
        return self.widths[0]

    @property
    def n_out(self):
        return self.widths[-1]

    @property
    def n_params(self):
        return sum(w.size for w in self.W)


@dataclasses.dataclass
class Mesh:
    X: np.ndarray           # float64 (V, 3) rest positions
    tets: np.ndarray        # int32 (T, 4), positively oriented
    vmass: np.ndarray       # float64 (V,) lumped vertex masses
    material: str = "stvk"  # stvk | neohookean
    E: float = 1e5
    nu: float = 0.4

    @property
    def n_vert(self):
        return self.X.shape[0]

    @property
    def n_tet(self):
        return self.tets.shape[0]


@dataclasses.dataclass
class State:
    qbar: np.ndarray        # float64 (r,)
    qbar_dot: np.ndarray    # float64 (r,)
    dt: float = 1.0 / 60.0


@dataclasses.dataclass
class Workload:
    name: str
    dec: Decoder
    mesh: Mesh
    cub_tets: np.ndarray    # int32 (C,) distinct tet indices
    cub_w: np.ndarray       # float32 (C,) weights in [0.5, 2]
    state: State
    f_ext: np.ndarray       # float32 (N,) external force (zeros or gravity)
    max_iter: int = 5


def make_decoder(widths, seed, act="tanh", out_scale=0.1, bias=True):
    """Xavier-normal weights, U(+-1/sqrt(fan_in)) biases; the output layer is
    scaled by ``out_scale`` so decoded displacements stay a fraction of the
    grid spacing (1.0) and no tet inverts.

    ``bias=False`` zeroes every bias (the weights are drawn from the same stream).
    With an odd activation (tanh, sin, linear) the decoder is then odd and
    D(0) = 0: the latent origin decodes to the rest shape, as it does for an
    autoencoder trained on poses around rest.  A decoder with random biases has
    no rest state in its range, so implicit-Euler frames that relax the elastic
    energy drive the latent toward tanh saturation (where J -> 0 and the reduced
    residual vanishes spuriously)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W, b = [], []
    L = len(widths) - 1
    for l in range(L):
        n_in, n_out = widths[l], widths[l + 1]
        std = np.sqrt(2.0 / (n_in + n_out))
        w = rng.standard_normal((n_out, n_in), dtype=np.float32) * np.float32(std)
        bb = rng.uniform(-1.0, 1.0, n_out).astype(np.float32) / np.float32(np.sqrt(n_in))
        if l == L - 1:
            w *= np.float32(out_scale)
            bb *= np.float32(out_scale)
        if not bias:
            bb[:] = 0.0
        W.append(np.ascontiguousarray(w))
        b.append(np.ascontiguousarray(bb))
    return Decoder(list(widths), W, b, act)


@dataclasses.dataclass
class WNet:
    widths: list            # [N, h1, h2, h3, n_tet]
    W: list                 # float32 (n_out, n_in)
    b: list                 # float32 (n_out,)


def make_wnet(n_in, n_tet, seed, hidden=(64, 64, 64), out_scale=0.3, out_bias=1.0):
    """Weight network with random weights: Xavier-normal layers n_in-h1-h2-h3-n_tet,
    U(+-1/sqrt(fan_in)) biases; the last layer scaled by ``out_scale`` with biases
    ``out_bias``, so the squared outputs sit around 1 (the range of the seeded
    cubature weights they replace)."""
    rng = np.random.Generator(np.random.PCG64(seed + 49979687))
    widths = [n_in] + list(hidden) + [n_tet]
    W, b = [], []
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        w = rng.standard_normal((fo, fi), dtype=np.float32) * np.float32(np.sqrt(2.0 / (fi + fo)))
        bb = rng.uniform(-1.0, 1.0, fo).astype(np.float32) / np.float32(np.sqrt(fi))
        if l == len(widths) - 2:
            w *= np.float32(out_scale)
            bb[:] = np.float32(out_bias)
        W.append(np.ascontiguousarray(w))
        b.append(np.ascontiguousarray(bb))
    return WNet(widths, W, b)


def make_linear_basis(N, n_p, seed):
    """Orthonormal N x n_p basis (unit, mutually orthogonal columns, as the paper's PCA
    basis): QR of a seeded Gaussian matrix.  float32."""
    rng = np.random.Generator(np.random.PCG64(seed + 86028121))
    Q, _ = np.linalg.qr(rng.standard_normal((N, n_p)))
    return np.ascontiguousarray(Q.astype(np.float32))


def make_linear_state(n_p, seed, p_std=0.5, pdot_std=0.1):
    """pbar ~ N(0, p_std^2), pbar_dot ~ N(0, pdot_std^2) (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed + 32452867))
    return rng.normal(0.0, p_std, n_p), rng.normal(0.0, pdot_std, n_p)


def make_grid_mesh(nx, ny, nz, seed, material="stvk", E=1e5, nu=0.4, spacing=1.0):
    """Regular vertex grid (nx*ny*nz vertices, spacing 1, origin 0), five tets
    per cube alternating with the parity of (i+j+k), positive orientation,
    lumped masses uniform in [0.5, 1.5]."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    X = np.stack([ii, jj, kk], -1).reshape(-1, 3).astype(np.float64) * spacing

    def vid(i, j, k):
        return (i * ny + j) * nz + k

    tets = []
    for i in range(nx - 1):
        for j in range(ny - 1):
            for k in range(nz - 1):
                def v(o):
                    return vid(i + o[0], j + o[1], k + o[2])
                par = (i + j + k) & 1
                cen = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
                oth = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
                if par:
                    cen, oth = oth, cen
                tets.append([v(o) for o in cen])
                for corner in oth:
                    nb = [o for o in cen if sum(abs(a - b) for a, b in zip(o, corner)) == 1]
                    tets.append([v(corner)] + [v(o) for o in nb])
    tets = np.asarray(tets, dtype=np.int32)
    # orient: det[x1-x0, x2-x0, x3-x0] > 0
    P = X[tets]
    D = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], -1)
    neg = np.linalg.det(D) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    vmass = rng.uniform(0.5, 1.5, X.shape[0])
    return Mesh(X, np.ascontiguousarray(tets), vmass, material, E, nu)


def make_cubature(n_tet, n_cub, seed, frame=0):
    """Distinct seeded cubature tets (fixed per workload) and weights uniform in
    [0.5, 2] (redrawn per frame: the frame index enters the weight stream)."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    idx = np.sort(rng.choice(n_tet, size=n_cub, replace=False)).astype(np.int32)
    wrng = np.random.Generator(np.random.PCG64([seed + 1299709, frame]))
    w = wrng.uniform(0.5, 2.0, n_cub).astype(np.float32)
    return idx, w


def make_state(r, seed, dt=1.0 / 60.0, q_std=0.5, qdot_std=0.1):
    """Latent state qbar ~ N(0, q_std^2), qbar_dot ~ N(0, qdot_std^2)."""
    rng = np.random.Generator(np.random.PCG64(seed + 15485863))
    return State(rng.normal(0.0, q_std, r), rng.normal(0.0, qdot_std, r), dt)


def gravity_force(vmass):
    f = np.zeros((vmass.shape[0], 3), dtype=np.float64)
    f[:, 1] = -GRAVITY * vmass
    return f.reshape(-1).astype(np.float32)


SMALL_WIDTHS = [5, 64, 256, 1024, 3000]
# Paper-scale initial latent spread.  With qbar ~ N(0, 0.5^2) in 30 dimensions the
# Neo-Hookean body starts so far from rest (cubature energy ~1e4) that a^T H
# dominates the Newton matrix and makes it indefinite; a start near rest keeps the
# implicit-Euler frames in the regime where Newton converges.
PAPER_Q_STD = 0.05
PAPER_WIDTHS = [30, 128, 256, 512, 1024, 2048, 2048, 2048, 4096, 4096, 60000]


def small(seed=1, act="tanh"):
    """Latent 5, 1000-vertex grid, StVK, 64 cubature tets, no external force;
    bias-free decoder (rest shape at q = 0)."""
    dec = make_decoder(SMALL_WIDTHS, seed, act, bias=False)
    mesh = make_grid_mesh(10, 10, 10, seed, "stvk", 1e5, 0.4)
    cub, w = make_cubature(mesh.n_tet, 64, seed)
    st = make_state(dec.r, seed)
    return Workload("small", dec, mesh, cub, w, st, np.zeros(dec.n_out, np.float32))


def paper(seed=2, act="tanh"):
    """Latent 30, ten-layer decoder onto a 20000-vertex grid, Neo-Hookean,
    500 cubature tets, gravity; bias-free decoder (rest shape at q = 0)."""
    dec = make_decoder(PAPER_WIDTHS, seed, act, bias=False)
    mesh = make_grid_mesh(20, 20, 50, seed, "neohookean", 5e5, 0.45)
    cub, w = make_cubature(mesh.n_tet, 500, seed)
    st = make_state(dec.r, seed, q_std=PAPER_Q_STD)
    return Workload("paper", dec, mesh, cub, w, st, gravity_force(mesh.vmass))


def medium(seed=2, act="tanh"):
    """The paper-scale decoder's hidden layers with a 20x20x17 grid (N = 20400 output
    DOFs, 160 output tiles, 334 MB of output-layer weights: larger than L2), for
    profiler captures that must stay small; material, cubature, gravity and start
    state as in ``paper``."""
    widths = PAPER_WIDTHS[:-1] + [3 * 20 * 20 * 17]
    dec = make_decoder(widths, seed, act, bias=False)
    mesh = make_grid_mesh(20, 20, 17, seed, "neohookean", 5e5, 0.45)
    cub, w = make_cubature(mesh.n_tet, 500, seed)
    st = make_state(dec.r, seed, q_std=PAPER_Q_STD)
    return Workload("medium", dec, mesh, cub, w, st, gravity_force(mesh.vmass))


STRING_HIDDEN = [32, 64, 128, 256, 256, 256, 256]
STRING_Q_STD = 0.1


def string_shapes(n_strings=320, seed=4, r_range=(3, 15), v_range=(200, 2000)):
    """Latent sizes r_s ~ U{r_range} and vertex counts V_s ~ U[v_range] (rounded down to a
    multiple of 4) of the strings made by ``strings`` with the same arguments."""
    rng = np.random.Generator(np.random.PCG64(seed + 32452843))
    rs = rng.integers(r_range[0], r_range[1] + 1, n_strings)
    vs = rng.integers(v_range[0], v_range[1] + 1, n_strings) // 4 * 4
    return [int(x) for x in rs], [int(x) for x in vs]


def string_widths(r, V):
    """Layer widths of a string's depth-8 decoder."""
    return [r] + STRING_HIDDEN + [3 * V]


def strings(n_strings=320, seed=4, act="tanh", r_range=(3, 15), v_range=(200, 2000),
            n_cub=32, only=None):
    """Substructured model of independent strings (the puffer ball's 320 strings): string
    s has latent r_s ~ U{r_range}, V_s ~ U[v_range] vertices (rounded down to a multiple
    of 4) on a 2 x 2 x V_s/4 grid, a bias-free depth-8 decoder
    r_s-32-64-128-256-256-256-256-3V_s, StVK (E = 1e5, nu = 0.4), ``n_cub`` cubature tets,
    start qbar ~ N(0, 0.1^2), qbar_dot ~ N(0, 0.1^2), no external force.  Returns a list of
    workloads (string s seeded from seed and s); ``only`` (indices) makes just those
    strings, each identical to its copy in the full list."""
    rs, vs = string_shapes(n_strings, seed, r_range, v_range)
    out = []
    for s in (range(n_strings) if only is None else only):
        r, V = rs[s], vs[s]
        ss = seed * 100003 + s
        dec = make_decoder(string_widths(r, V), ss, act, bias=False)
        mesh = make_grid_mesh(2, 2, V // 4, ss, "stvk", 1e5, 0.4)
        cub, w = make_cubature(mesh.n_tet, n_cub, ss)
        st = make_state(r, ss, q_std=STRING_Q_STD)
        out.append(Workload("string%d" % s, dec, mesh, cub, w, st, np.zeros(dec.n_out, np.float32)))
    return out


@dataclasses.dataclass
class Coupled:
    """Substructured body: domains joined at interfaces.  A row (d, i, e, j) of
    ``pairs`` says vertex i of domain d and vertex j of domain e coincide at rest; a
    row (d, i) of ``anchors`` holds vertex i of domain d at its rest position; ``k_c``
    is the stiffness of both ties; ``parents[d]`` is the domain d hangs from (-1 for
    an anchored root)."""
    domains: list
    parents: list
    pairs: np.ndarray       # int32 (P, 4)
    anchors: np.ndarray     # int32 (Q, 2)
    k_c: float


def string_faces(V):
    """Vertex ids of the base face (k = 0) and the tip face (k = V/4 - 1) of a
    2 x 2 x V/4 string grid, in the same (i, j) order."""
    nz = V // 4
    base = [(i * 2 + j) * nz for i in range(2) for j in range(2)]
    return base, [b + nz - 1 for b in base]


def coupled_strings(parents, seed=6, r=3, V=16, hidden=(16, 32), act="tanh", bias=False,
                    out_scale=0.1, material="stvk", E=1e5, nu=0.4, k_c=1e5, n_cub=8,
                    q_std=0.05, gravity=True):
    """Strings joined into a tree (the cactus's domain hierarchy; a chain is a tree
    with one child per domain): domain d is a 2 x 2 x V/4 string with decoder
    r-hidden-3V, and its base face coincides at rest with the tip face of domain
    parents[d] (a root's base face is anchored).  Bias-free decoders by default, so
    every domain is at rest at its latent origin and the ties start slack there.
    Seeded per domain from seed and d."""
    base, tip = string_faces(V)
    domains, pairs, anchors = [], [], []
    for d, p in enumerate(parents):
        ss = seed * 100003 + d
        dec = make_decoder([r, *hidden, 3 * V], ss, act, out_scale=out_scale, bias=bias)
        mesh = make_grid_mesh(2, 2, V // 4, ss, material, E, nu)
        cub, w = make_cubature(mesh.n_tet, min(n_cub, mesh.n_tet), ss)
        st = make_state(r, ss, q_std=q_std)
        f = gravity_force(mesh.vmass) if gravity else np.zeros(dec.n_out, np.float32)
        domains.append(Workload("domain%d" % d, dec, mesh, cub, w, st, f))
        if p < 0:
            anchors += [(d, b) for b in base]
        else:
            assert p < d, "a parent precedes its children"
            pairs += [(d, b, p, t) for b, t in zip(base, tip)]
    return Coupled(domains, list(parents), np.asarray(pairs, np.int32).reshape(-1, 4),
                   np.asarray(anchors, np.int32).reshape(-1, 2), float(k_c))


def custom(widths, grid, n_cub, seed, act="tanh", material="stvk", E=1e5, nu=0.4,
           gravity=False):
    """Arbitrary-shape workload for parity sweeps; ``widths[-1]`` must equal
    3 * prod(grid)."""
    assert widths[-1] == 3 * grid[0] * grid[1] * grid[2]
    dec = make_decoder(widths, seed, act)
    mesh = make_grid_mesh(*grid, seed, material, E, nu)
    cub, w = make_cubature(mesh.n_tet, min(n_cub, mesh.n_tet), seed)
    st = make_state(dec.r, seed)
    f = gravity_force(mesh.vmass) if gravity else np.zeros(dec.n_out, np.float32)
    return Workload("custom", dec, mesh, cub, w, st, f)


def newton_start(state):
    """Initial Newton iterate q0 = qbar + dt * qbar_dot (so (q0-qbar)/dt = qbar_dot)."""
    return state.qbar + state.dt * state.qbar_dot
