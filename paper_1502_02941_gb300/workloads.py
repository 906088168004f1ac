"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds problem DATA only (meshes, coefficients, manufactured
solutions and the source/boundary data derived from them by calculus); it
contains none of the DG method's arithmetic.  Functions are written against an
array namespace ``xp`` (numpy or torch) so the same formulas serve host and
device inputs.

Meshes follow the data layout of Sec. 2.1 of Uzunca & Karasozen
(arXiv:1502.02941): Nodes [nv,2], Elements [ne,3] counter-clockwise,
Dirichlet/Neumann [.,2] start/end node of each boundary edge -- 0-based here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

# The initial mesh printed in Sec. 2.1 (Fig. 2), converted to 0-based indices.
FIXTURE_NODES = np.array([[0, 0], [0.5, 0], [1, 0], [0, 0.5], [0.5, 0.5], [1, 0.5],
                          [0, 1], [0.5, 1], [1, 1]], dtype=np.float64)
FIXTURE_ELEMS = np.array([[4, 1, 5], [1, 2, 5], [5, 2, 6], [2, 3, 6], [7, 4, 8], [4, 5, 8],
                          [8, 5, 9], [5, 6, 9]], dtype=np.int32) - 1
FIXTURE_DIRICHLET = np.array([[1, 2], [2, 3], [1, 4], [3, 6], [4, 7], [6, 9], [7, 8], [8, 9]],
                             dtype=np.int32) - 1


@dataclass
class MeshArrays:
    nodes: np.ndarray
    elems: np.ndarray
    dirichlet: np.ndarray
    neumann: np.ndarray

    @property
    def ne(self):
        return int(self.elems.shape[0])


def structured_mesh(N: int, neumann_sides=(), x0=0.0, y0=0.0, L=1.0) -> MeshArrays:
    """N x N squares on [x0,x0+L]x[y0,y0+L], each split by its "/" diagonal
    into an upper-left and a lower-right triangle, counter-clockwise, in the
    element order of the paper's Fig. 2 (row by row, upper then lower).

    neumann_sides: subset of {"left","right","bottom","top"}; the rest are
    Dirichlet."""
    h = L / N
    xs = x0 + np.arange(N + 1) * h
    ys = y0 + np.arange(N + 1) * h
    X, Y = np.meshgrid(xs, ys)           # node (i,j) -> j*(N+1)+i
    nodes = np.stack([X.ravel(), Y.ravel()], 1)
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    i = i.ravel(); j = j.ravel()
    a = j * (N + 1) + i                  # (i, j)
    b = a + 1                            # (i+1, j)
    c = a + (N + 1)                      # (i, j+1)
    d = c + 1                            # (i+1, j+1)
    upper = np.stack([c, a, d], 1)
    lower = np.stack([a, b, d], 1)
    elems = np.stack([upper, lower], 1).reshape(-1, 3).astype(np.int32)
    r = np.arange(N)
    sides = {
        "bottom": np.stack([r, r + 1], 1),
        "right": np.stack([r * (N + 1) + N, (r + 1) * (N + 1) + N], 1),
        "top": np.stack([N * (N + 1) + r + 1, N * (N + 1) + r], 1),
        "left": np.stack([(r + 1) * (N + 1), r * (N + 1)], 1),
    }
    dl = [sides[s] for s in ("bottom", "right", "top", "left") if s not in neumann_sides]
    nl = [sides[s] for s in ("bottom", "right", "top", "left") if s in neumann_sides]
    dirichlet = np.concatenate(dl).astype(np.int32) if dl else np.zeros((0, 2), np.int32)
    neumann = np.concatenate(nl).astype(np.int32) if nl else np.zeros((0, 2), np.int32)
    return MeshArrays(nodes, elems, dirichlet, neumann)


def lshape_mesh() -> MeshArrays:
    """An L-shaped polygon: the unit square without its upper-right quarter, as
    six triangles of the 2x2 split-square mesh.  Dirichlet on the edges that
    touch x = 0 or y = 0, Neumann on the rest; boundary edges counter-clockwise."""
    m = structured_mesh(2)
    keep = [K for K in range(m.ne) if not (m.nodes[m.elems[K]].mean(0) > 0.5).all()]
    elems = m.elems[keep].astype(np.int32)
    count: dict = {}
    for t in elems:
        for f in range(3):
            e = tuple(sorted((int(t[f]), int(t[(f + 1) % 3]))))
            count[e] = count.get(e, 0) + 1
    bnd = [(int(t[f]), int(t[(f + 1) % 3])) for t in elems for f in range(3)
           if count[tuple(sorted((int(t[f]), int(t[(f + 1) % 3]))))] == 1]
    on_axis = lambda e: (m.nodes[list(e)] == 0.0).any()   # noqa: E731
    dirichlet = np.array([e for e in bnd if on_axis(e)], np.int32).reshape(-1, 2)
    neumann = np.array([e for e in bnd if not on_axis(e)], np.int32).reshape(-1, 2)
    return MeshArrays(m.nodes, elems, dirichlet, neumann)


def perturbed_mesh(N: int, seed: int, amount: float = 0.2, neumann_sides=()) -> MeshArrays:
    """structured_mesh with interior nodes moved by up to amount*h (seeded):
    a general unstructured-looking triangulation that stays valid."""
    m = structured_mesh(N, neumann_sides)
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    nodes = m.nodes.copy()
    interior = (nodes[:, 0] > 0) & (nodes[:, 0] < 1) & (nodes[:, 1] > 0) & (nodes[:, 1] < 1)
    nodes[interior] += rng.uniform(-amount * h, amount * h, size=(interior.sum(), 2))
    return MeshArrays(nodes, m.elems, m.dirichlet, m.neumann)


# ---------------------------------------------------------------------------
# problems: coefficients + exact solution (u, grad u, laplacian u)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """alpha u - eps Lap u + b.grad u (+ r(u)) = f with eps, alpha constant and
    b(x,y) = (b0 + b1 x + b2 y, b3 + b4 x + b5 y) (Eq. (1)); with reaction =
    (p, c) the non-linear reaction r(u) = c u^p of Sec. 3 is part of the
    model (Eq. (nonlin))."""
    name: str
    eps: float
    alpha: float
    b: tuple
    exact: object = None          # callable(xp, x, y) -> (u, ux, uy, lap)
    source: object = None         # callable(xp, x, y) -> f, when there is no exact solution
    neumann_sides: tuple = ()
    meta: dict = field(default_factory=dict)
    reaction: tuple = ()          # (p, c): r(u) = c u^p
    # variable diffusion coefficient, the paper's fdiff(x, y) (Sec. 2.2):
    # callable(xp, x, y) -> (eps, eps_x, eps_y); None = the constant eps
    eps_fn: object = None

    def eps_at(self, xp, x, y):
        """The diffusion coefficient at points (the constant, or eps_fn)."""
        if self.eps_fn is None:
            return self.eps + 0.0 * x
        return self.eps_fn(xp, x, y)[0]

    def bvec(self, xp, x, y):
        b = self.b
        return b[0] + b[1] * x + b[2] * y, b[3] + b[4] * x + b[5] * y

    def f(self, xp, x, y):
        """f = alpha u - eps Lap u + b.grad u from the exact solution."""
        if self.exact is None:
            return self.source(xp, x, y)
        u, ux, uy, lap = self.exact(xp, x, y)
        bx, by = self.bvec(xp, x, y)
        if self.eps_fn is None:
            f = self.alpha * u - self.eps * lap + bx * ux + by * uy
        else:   # -div(eps grad u) = -eps Lap u - grad eps . grad u
            e, ex_, ey_ = self.eps_fn(xp, x, y)
            f = self.alpha * u - e * lap - (ex_ * ux + ey_ * uy) + bx * ux + by * uy
        if self.reaction:
            p, c = self.reaction
            f = f + c * u ** p
        return f

    def u(self, xp, x, y):
        if self.exact is None:
            return None
        return self.exact(xp, x, y)[0]

    def gD(self, xp, x, y):
        """Dirichlet data (the exact solution; zero without one)."""
        if self.exact is None:
            return 0.0 * x
        return self.exact(xp, x, y)[0]

    def gN(self, xp, x, y, nx, ny):
        """Neumann data eps grad u . n (Eq. (1c))."""
        if self.exact is None:
            return 0.0 * x
        _, ux, uy, _ = self.exact(xp, x, y)
        return self.eps_at(xp, x, y) * (ux * nx + uy * ny)


def sinsin(xp, x, y):
    """u = sin(pi x) sin(pi y)."""
    s, c = xp.sin, xp.cos
    pi = math.pi
    u = s(pi * x) * s(pi * y)
    return u, pi * c(pi * x) * s(pi * y), pi * s(pi * x) * c(pi * y), -2 * pi * pi * u


def boundary_layer(eps):
    """u = x y (1 - exp((x-1)/eps)) (1 - exp((y-1)/eps))."""
    def ex(xp, x, y):
        E1 = xp.exp((x - 1.0) / eps)
        E2 = xp.exp((y - 1.0) / eps)
        X = x * (1 - E1); Y = y * (1 - E2)
        Xp = 1 - E1 - x / eps * E1
        Yp = 1 - E2 - y / eps * E2
        Xpp = -(2.0 / eps + x / eps ** 2) * E1
        Ypp = -(2.0 / eps + y / eps ** 2) * E2
        return X * Y, Xp * Y, X * Yp, Xpp * Y + X * Ypp
    return ex


def gaussian_bump(xp, x, y):
    """u = exp(-50((x-0.5)^2 + (y-0.3)^2))."""
    dx = x - 0.5; dy = y - 0.3
    u = xp.exp(-50.0 * (dx * dx + dy * dy))
    ux = -100.0 * dx * u; uy = -100.0 * dy * u
    lap = (-100.0 + 1e4 * dx * dx) * u + (-100.0 + 1e4 * dy * dy) * u
    return u, ux, uy, lap


def tanh_layer(eps):
    """The paper's example solution u = (1 - tanh((2x - y - 0.25)/sqrt(5 eps)))/2
    (Sec. 2.2 and the listing's fexact)."""
    s5 = math.sqrt(5.0 * eps)
    def ex(xp, x, y):
        z = (2 * x - y - 0.25) / s5
        t = xp.tanh(z)
        sech2 = 1 - t * t
        u = 0.5 * (1 - t)
        ux = -sech2 / s5
        uy = 0.5 * sech2 / s5
        lap = (0.8 / eps) * t * sech2 + (0.2 / eps) * t * sech2
        return u, ux, uy, lap
    return ex


def polynomial(a: int, bexp: int, c0=0.3):
    """u = c0 + x^a y^b (degree a+b), for exact-reproduction checks."""
    def ex(xp, x, y):
        u = c0 + x ** a * y ** bexp
        ux = a * x ** (a - 1) * y ** bexp if a > 0 else 0.0 * x
        uy = bexp * x ** a * y ** (bexp - 1) if bexp > 0 else 0.0 * x
        uxx = a * (a - 1) * x ** (a - 2) * y ** bexp if a > 1 else 0.0 * x
        uyy = bexp * (bexp - 1) * x ** a * y ** (bexp - 2) if bexp > 1 else 0.0 * x
        return u, ux, uy, uxx + uyy
    return ex


def affine_eps(e0, e1, e2):
    """eps(x, y) = e0 + e1 x + e2 y (with its gradient)."""
    def fn(xp, x, y):
        return e0 + e1 * x + e2 * y, e1 + 0.0 * x, e2 + 0.0 * x
    return fn


def wavy_eps(e0=1.0, amp=0.5):
    """eps(x, y) = e0 + amp sin(2 pi x) cos(pi y) (with its gradient); positive
    for amp < e0."""
    pi = math.pi

    def fn(xp, x, y):
        s2, c2 = xp.sin(2 * pi * x), xp.cos(2 * pi * x)
        cy, sy = xp.cos(pi * y), xp.sin(pi * y)
        return e0 + amp * s2 * cy, amp * 2 * pi * c2 * cy, -amp * pi * s2 * sy
    return fn


def gaussians_source(centres, widths, amp=1.0):
    """f = sum_i amp exp(-|x - c_i|^2 / (2 w_i^2))."""
    def src(xp, x, y):
        f = 0.0 * x
        for (cx, cy), w in zip(centres, widths):
            f = f + amp * xp.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))
        return f
    return src


# ---------------------------------------------------------------------------
# the workloads: sine 8x8 P1, boundary layer P2, Gaussian bump P3, and the
# random families of the batched and learned solves
# ---------------------------------------------------------------------------

@dataclass
class Config:
    name: str
    N: int
    k: int
    method: int            # 1 NIPG, 2 SIPG, 3 IIPG
    problem: Problem
    sigma: float | None = None   # interior penalty override; boundary = 2 sigma


def sine_8x8() -> Config:
    """8x8 split squares (128 triangles), P1, SIPG sigma = 6k^2, eps=1, b=0,
    alpha=0, all Dirichlet, u = sin(pi x) sin(pi y); direct solve."""
    return Config("sine_sipg_p1_n8", 8, 1, 2, Problem("sinsin", 1.0, 0.0, (0, 0, 0, 0, 0, 0), sinsin),
                  sigma=6.0)


def boundary_layer_p2(method: int = 2, N: int = 256) -> Config:
    """256x256 split squares (131072 triangles), P2, NIPG or SIPG, eps=1e-6,
    b=(1,0), alpha=1, boundary-layer solution, all Dirichlet; GMRES(50)+BJ."""
    eps = 1e-6
    return Config(f"layer_{'nipg' if method == 1 else 'sipg'}_p2_n{N}", N, 2, method,
                  Problem("boundary_layer", eps, 1.0, (1.0, 0, 0, 0, 0, 0), boundary_layer(eps)))


def gaussian_bump_p3(N: int = 512) -> Config:
    """512x512 split squares (524288 triangles), P3, SIPG, eps=1e-3,
    b=(0.5-y, x-0.5), alpha=0.1, Gaussian-bump solution; Dirichlet on
    left/bottom, Neumann on right/top; mixed precision."""
    return Config(f"bump_sipg_p3_n{N}", N, 3, 2,
                  Problem("gaussian", 1e-3, 0.1, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), gaussian_bump,
                          neumann_sides=("right", "top")))


def tanh_nonlinear(N: int = 8, k: int = 1, method: int = 2) -> Config:
    """The paper's non-linear example (Sec. 3 and its Main_Nonlinear listing):
    the initial mesh refined twice (8x8 split squares, 128 triangles), SIPG P1,
    eps = 1e-6, b = (1, 2)/sqrt(5), alpha = 1, r(u) = u^2, Dirichlet data on all
    sides from u = (1 - tanh((2x - y - 0.25)/sqrt(5 eps)))/2."""
    eps = 1e-6
    s5 = 1.0 / math.sqrt(5.0)
    return Config(f"tanh_nl_{'nipg' if method == 1 else ('sipg' if method == 2 else 'iipg')}_p{k}_n{N}", N, k,
                  method, Problem("tanh_layer_u2", eps, 1.0, (s5, 0, 0, 2 * s5, 0, 0), tanh_layer(eps),
                                  reaction=(2, 1.0)))


# seed of instance i of a random family: SEED_BASE[family] + i
SEED_BASE = {"batched": 20264000, "learned": 20265000}


def instance_seed(family: str, instance: int) -> int:
    return SEED_BASE[family] + instance


def random_instance(family: str, instance: int, N_range=(16, 128), k_choices=(1, 2),
                    N_fixed: int | None = None, k_fixed: int | None = None) -> Config:
    """Per-instance draw for the batched and learned workloads: N uniform in
    N_range, k from k_choices, eps log-uniform on [1e-6,1e-1], b = U[0,1] times
    a unit vector at a U[0,2pi) angle, alpha ~ U[0,1], f a sum of 4 Gaussians
    (centres U[0,1]^2, widths U[0.05,0.2], amplitude 1); SIPG, homogeneous
    Dirichlet data on all sides."""
    rng = np.random.default_rng(instance_seed(family, instance))
    N = int(rng.integers(N_range[0], N_range[1] + 1)) if N_fixed is None else N_fixed
    k = int(rng.choice(k_choices)) if k_fixed is None else k_fixed
    eps = float(10 ** rng.uniform(-6, -1))
    theta = rng.uniform(0, 2 * np.pi)
    s = rng.uniform(0, 1)
    alpha = float(rng.uniform(0, 1))
    centres = rng.uniform(0, 1, size=(4, 2))
    widths = rng.uniform(0.05, 0.2, size=4)
    prob = Problem("gaussians", eps, alpha, (s * np.cos(theta), 0, 0, s * np.sin(theta), 0, 0),
                   None, gaussians_source([tuple(c) for c in centres], list(widths)))
    return Config(f"{family}_inst{instance}", N, k, 2, prob)


def batch_by_degree(family: str, n_inst: int, N_range=(16, 128)):
    """Instances 0..n_inst-1 of the batched workload grouped by their degree:
    {k: (cfgs, mesh, elem_start, coeffs)}, one batch per degree (a batch shares
    k), each instance keeping its own draw."""
    groups: dict[int, list] = {}
    for i in range(n_inst):
        c = random_instance(family, i, N_range=N_range)
        groups.setdefault(c.k, []).append(c)
    out = {}
    for k in sorted(groups):
        cfgs = groups[k]
        ma, starts = concat_meshes([structured_mesh(c.N) for c in cfgs])
        coeffs = np.array([[c.problem.eps, c.problem.alpha, *c.problem.b] for c in cfgs])
        out[k] = (cfgs, ma, starts, coeffs)
    return out


def concat_meshes(meshes):
    """Concatenate independent meshes into one (node and element ids offset);
    returns the MeshArrays and elem_start [len+1] (instance i owns elements
    elem_start[i]..elem_start[i+1]-1)."""
    nodes, elems, dirs, neus, starts = [], [], [], [], [0]
    off = 0
    for m in meshes:
        nodes.append(m.nodes)
        elems.append(m.elems + off)
        dirs.append(m.dirichlet + off)
        neus.append(m.neumann + off)
        off += m.nodes.shape[0]
        starts.append(starts[-1] + m.elems.shape[0])
    return (MeshArrays(np.concatenate(nodes), np.concatenate(elems).astype(np.int32),
                       np.concatenate(dirs).astype(np.int32),
                       np.concatenate(neus).astype(np.int32) if neus else np.zeros((0, 2), np.int32)),
            np.array(starts, np.int32))


def batch(family: str, n_inst: int, k: int | None = None, N_fixed: int | None = None, N_range=(16, 128)):
    """Instances of the batched ("batched") or learned ("learned") workload
    with degree k (instances of the other degree are skipped, so that one batch
    shares k), their concatenated mesh, elem_start and coefficient table."""
    cfgs, i = [], 0
    while len(cfgs) < n_inst:
        c = random_instance(family, i, N_range=N_range, N_fixed=N_fixed)
        i += 1
        if k is not None and c.k != k:
            continue
        cfgs.append(c)
    meshes = [structured_mesh(c.N) for c in cfgs]
    ma, starts = concat_meshes(meshes)
    coeffs = np.array([[c.problem.eps, c.problem.alpha, *c.problem.b] for c in cfgs])
    return cfgs, ma, starts, coeffs
