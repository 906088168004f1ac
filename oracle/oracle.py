"""Python driver for the FP64 CPU oracle in ``dg_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use this module; the product library never does.
It shares no code with the CUDA path.  Everything here is argument marshalling
around the C routines, plus assembly of their block output into scipy sparse
matrices (a storage primitive) for the self-tests.

Paper: Uzunca & Karasozen, "A Matlab Tutorial for Diffusion-Convection-Reaction
Equations using DGFEM", arXiv:1502.02941.  Section / equation references in the
docstrings below are to that paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}
_use_omp = False

NIPG, SIPG, IIPG = 1, 2, 3   # the paper's `method` numbering (Sec. 2.2)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile dg_oracle.c into liboracle.so with gcc (portable flags only).
    openmp=True builds liboracle_omp.so, the same source with its OpenMP loops
    switched on, used only to time the oracle on all host cores."""
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        extra = ["-DORC_OPENMP", "-fopenmp"] if openmp else []
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", *extra,
               "-o", lib + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(lib + ".tmp", lib)
    return lib


def set_openmp(on: bool) -> None:
    """Route later oracle calls to the all-cores timing build (True) or the
    serial build (False, the default and what every test uses)."""
    global _use_omp
    _use_omp = bool(on)


def num_threads() -> int:
    """Host threads the current build's loops run on."""
    return int(_load().orc_num_threads())


def _load():
    key = "omp" if _use_omp else "serial"
    if key not in _libs:
        path = build(openmp=_use_omp)
        _libs[key] = ctypes.CDLL(path)
    return _libs[key]


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _d(a):
    return _p(a, ctypes.c_double)


def _i(a):
    return _p(a, ctypes.c_int)


def set_parameter(method: int, degree: int):
    """(sigma_interior, kappa) as chosen in Sec. 1 (last paragraph) and the
    listing's set_parameter (Sec. 4): NIPG kappa=+1, sigma=1; SIPG kappa=-1,
    IIPG kappa=0, both sigma=3k(k+1).  Boundary edges use twice sigma."""
    if method == NIPG:
        return 1.0, 1.0
    if method == SIPG:
        return 3.0 * degree * (degree + 1), -1.0
    if method == IIPG:
        return 3.0 * degree * (degree + 1), 0.0
    raise ValueError("method must be 1 (NIPG), 2 (SIPG) or 3 (IIPG)")


def nbasis(k: int) -> int:
    """Unknowns per element, (k+1)(k+2)/2 (the listing's DoF formula, Sec. 4)."""
    return (k + 1) * (k + 2) // 2


def gauss_legendre01(n: int):
    lib = _load()
    t = np.zeros(n)
    w = np.zeros(n)
    lib.orc_gauss_legendre01(ctypes.c_int(n), _d(t), _d(w))
    return t, w


@dataclass
class Mesh:
    """Mesh arrays of Sec. 2.1 (0-based) plus the oracle's edge table."""
    nodes: np.ndarray       # [nv,2] float64
    elems: np.ndarray       # [ne,3] int32, counter-clockwise
    dirichlet: np.ndarray   # [nd,2] int32
    neumann: np.ndarray     # [nn,2] int32
    edges: np.ndarray       # [ned,5] int32: va, vb, Ki, Kj(-1 bdry), type(0/1/2)
    elem_edges: np.ndarray  # [ne,3] int32

    @property
    def ne(self):
        return self.elems.shape[0]

    @property
    def ned(self):
        return self.edges.shape[0]

    @property
    def n_bedges(self):
        return int((self.edges[:, 3] < 0).sum())

    @property
    def n_interior(self):
        return int((self.edges[:, 3] >= 0).sum())


MESH_ERRORS = {-1: "element not counter-clockwise", -2: "edge shared by more than two elements",
               -3: "boundary edge without boundary condition", -4: "node index out of range"}


def _arrays(nodes, elems, dirichlet, neumann):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 2)
    elems = np.ascontiguousarray(elems, dtype=np.int32).reshape(-1, 3)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.int32).reshape(-1, 2)
    neumann = np.ascontiguousarray(neumann, dtype=np.int32).reshape(-1, 2)
    return nodes, elems, dirichlet, neumann


def make_mesh(nodes, elems, dirichlet, neumann) -> Mesh:
    """The paper's getmesh (Sec. 2.1): build the edge skeleton."""
    lib = _load()
    nodes, elems, dirichlet, neumann = _arrays(nodes, elems, dirichlet, neumann)
    ne = elems.shape[0]
    edges = np.zeros((3 * ne, 5), np.int32)
    ee = np.zeros((ne, 3), np.int32)
    ned = lib.orc_edges(nodes.shape[0], _d(nodes), ne, _i(elems), dirichlet.shape[0], _i(dirichlet),
                        neumann.shape[0], _i(neumann), _i(edges), _i(ee))
    if ned < 0:
        raise ValueError(MESH_ERRORS.get(ned, f"mesh error {ned}"))
    return Mesh(nodes, elems, dirichlet, neumann, edges[:ned].copy(), ee)


def refine(nodes, elems, dirichlet, neumann):
    """The paper's uniformrefine (Sec. 2.1): one red refinement."""
    lib = _load()
    nodes, elems, dirichlet, neumann = _arrays(nodes, elems, dirichlet, neumann)
    ne = elems.shape[0]
    nv = nodes.shape[0]
    nodes_out = np.zeros((nv + 3 * ne, 2))
    elems_out = np.zeros((4 * ne, 3), np.int32)
    dir_out = np.zeros((2 * dirichlet.shape[0], 2), np.int32)
    neu_out = np.zeros((2 * neumann.shape[0], 2), np.int32)
    nv_new = lib.orc_refine(nv, _d(nodes), ne, _i(elems), dirichlet.shape[0], _i(dirichlet),
                            neumann.shape[0], _i(neumann), _d(nodes_out), _i(elems_out),
                            _i(dir_out), _i(neu_out))
    if nv_new < 0:
        raise ValueError(MESH_ERRORS.get(nv_new, f"mesh error {nv_new}"))
    return nodes_out[:nv_new].copy(), elems_out, dir_out, neu_out


VOLUME, BOUNDARY, ERROR, EDGES = 0, 1, 2, 3


def quad_points(mesh: Mesh, k: int, which: int) -> np.ndarray:
    """Physical quadrature points (reading A-8): VOLUME [ne,(k+2)^2,2],
    BOUNDARY [n_bedges,k+2,2] (boundary edges in edge-table order, each run
    counter-clockwise for its element), ERROR [ne,(k+4)^2,2], EDGES
    [ned,k+2,2] (every edge in edge-table order, run from its first to its
    second node)."""
    lib = _load()
    if which == VOLUME:
        shape = (mesh.ne, (k + 2) ** 2, 2)
    elif which == BOUNDARY:
        shape = (mesh.n_bedges, k + 2, 2)
    elif which == EDGES:
        shape = (mesh.ned, k + 2, 2)
    else:
        shape = (mesh.ne, (k + 4) ** 2, 2)
    out = np.zeros(shape)
    lib.orc_quad_points(which, k, _d(mesh.nodes), mesh.ne, _i(mesh.elems), mesh.ned,
                        _i(mesh.edges), _d(out))
    return out


def boundary_normals(mesh: Mesh) -> np.ndarray:
    """Outward unit normal of each boundary edge (edge-table order)."""
    b = mesh.edges[mesh.edges[:, 3] < 0]
    d = mesh.nodes[b[:, 1]] - mesh.nodes[b[:, 0]]
    ln = np.sqrt((d ** 2).sum(1))
    return np.stack([d[:, 1] / ln, -d[:, 0] / ln], 1)


def boundary_types(mesh: Mesh) -> np.ndarray:
    return mesh.edges[mesh.edges[:, 3] < 0, 4].copy()


@dataclass
class System:
    k: int
    D_diag: np.ndarray
    D_off: np.ndarray
    C_diag: np.ndarray
    C_off: np.ndarray
    R_diag: np.ndarray
    R_off: np.ndarray
    F: np.ndarray

    @property
    def A_diag(self):
        return self.D_diag + self.C_diag + self.R_diag

    @property
    def A_off(self):
        return self.D_off + self.C_off + self.R_off


def assemble(mesh: Mesh, k: int, kappa: float, sigma_int: float, sigma_bdry: float,
             eps: float, alpha: float, b_affine, f_q, gD_q, gN_q,
             literal_rhs: bool = False, split: bool = True, b0: float = 1.0,
             eps_vol=None, eps_edge=None) -> System:
    """The paper's global_system (Sec. 2.3): D, C, R and F of Eq. (system).

    b_affine = (c0..c5): b(x,y) = (c0 + c1 x + c2 y, c3 + c4 x + c5 y).
    b0: the superpenalisation exponent of set_parameter (Sec. 4): the penalty
    terms carry sigma eps / |e|^b0 (reading A-3; the paper's default is 1).
    f_q at quad_points(VOLUME); gD_q, gN_q at quad_points(BOUNDARY) (gD is read
    on Dirichlet edges and on the inflow part of every boundary edge, reading
    A-6; gN on Neumann edges).  With split=False only A = D+C+R is stored (in
    D_*; C_* and R_* alias it).
    eps_vol / eps_edge: a variable diffusion coefficient (the paper's fdiff,
    Sec. 2.2) given at quad_points(VOLUME) [ne][(k+2)^2] and at
    quad_points(EDGES) [ned][k+2]; both or neither (then eps is the constant).
    """
    lib = _load()
    nb = nbasis(k)
    ne, ned = mesh.ne, mesh.ned
    b = np.ascontiguousarray(b_affine, dtype=np.float64).reshape(6)
    f_q = np.ascontiguousarray(f_q, dtype=np.float64).reshape(ne, (k + 2) ** 2)
    nbe = mesh.n_bedges
    gD_q = np.ascontiguousarray(gD_q if gD_q is not None else np.zeros((nbe, k + 2)), dtype=np.float64).reshape(nbe, k + 2)
    gN_q = np.ascontiguousarray(gN_q if gN_q is not None else np.zeros((nbe, k + 2)), dtype=np.float64).reshape(nbe, k + 2)
    if (eps_vol is None) != (eps_edge is None):
        raise ValueError("eps_vol and eps_edge are given together")
    if eps_vol is not None:
        eps_vol = np.ascontiguousarray(eps_vol, dtype=np.float64).reshape(ne, (k + 2) ** 2)
        eps_edge = np.ascontiguousarray(eps_edge, dtype=np.float64).reshape(ned, k + 2)
    Dd = np.zeros((ne, nb, nb))
    Do = np.zeros((ned, 2, nb, nb))
    if split:
        Cd, Co = np.zeros_like(Dd), np.zeros_like(Do)
        Rd, Ro = np.zeros_like(Dd), np.zeros_like(Do)
    else:
        Cd, Co, Rd, Ro = Dd, Do, Dd, Do
    F = np.zeros((ne, nb))
    lib.orc_assemble(k, _d(mesh.nodes), ne, _i(mesh.elems), ned, _i(mesh.edges), _i(mesh.elem_edges),
                     ctypes.c_double(kappa), ctypes.c_double(sigma_int), ctypes.c_double(sigma_bdry),
                     ctypes.c_double(eps), ctypes.c_double(alpha), _d(b), ctypes.c_int(int(literal_rhs)), ctypes.c_double(b0),
                     _d(f_q), _d(gD_q), _d(gN_q), _d(eps_vol), _d(eps_edge),
                     _d(Dd), _d(Do), _d(Cd), _d(Co), _d(Rd), _d(Ro), _d(F))
    if not split:
        z_d, z_o = np.zeros_like(Dd), np.zeros_like(Do)
        return System(k, Dd, Do, z_d, z_o, z_d, z_o, F.reshape(-1))
    return System(k, Dd, Do, Cd, Co, Rd, Ro, F.reshape(-1))


def to_sparse(mesh: Mesh, diag: np.ndarray, off: np.ndarray):
    """Global sparse matrix from the oracle's block storage (scipy CSR)."""
    import scipy.sparse as sp
    ne, nb = diag.shape[0], diag.shape[1]
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(nb), np.arange(nb), indexing="ij")
    for K in range(ne):
        rows.append(K * nb + ii.ravel()); cols.append(K * nb + jj.ravel()); vals.append(diag[K].ravel())
    for e in range(mesh.ned):
        Ki, Kj = mesh.edges[e, 2], mesh.edges[e, 3]
        if Kj < 0:
            continue
        rows.append(Ki * nb + ii.ravel()); cols.append(Kj * nb + jj.ravel()); vals.append(off[e, 0].ravel())
        rows.append(Kj * nb + ii.ravel()); cols.append(Ki * nb + jj.ravel()); vals.append(off[e, 1].ravel())
    n = ne * nb
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def apply(mesh: Mesh, diag, off, x):
    """y = (D+C+R) x on the block storage."""
    lib = _load()
    nb = diag.shape[1]
    diag = np.ascontiguousarray(diag); off = np.ascontiguousarray(off)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    y = np.zeros_like(x)
    lib.orc_apply(nb, mesh.ne, mesh.ned, _i(mesh.edges), _d(diag), _d(off), _d(x), _d(y))
    return y


def block_jacobi(diag):
    """Inverses of the diagonal blocks (Gauss-Jordan, partial pivoting)."""
    lib = _load()
    ne, nb = diag.shape[0], diag.shape[1]
    inv = np.zeros_like(diag)
    rc = lib.orc_block_jacobi(nb, ne, _d(np.ascontiguousarray(diag)), _d(inv))
    if rc != 0:
        raise ZeroDivisionError(f"singular diagonal block at element {-rc - 1}")
    return inv


def gmres(mesh: Mesh, diag, off, b, m=50, tol=1e-10, max_it=10000, precond=True):
    """Restarted GMRES(m) with right block-Jacobi preconditioning, x0 = 0.
    Returns (x, iterations, relres, converged)."""
    lib = _load()
    nb = diag.shape[1]
    diag = np.ascontiguousarray(diag); off = np.ascontiguousarray(off)
    inv = block_jacobi(diag) if precond else None
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b)
    info = np.zeros(2)
    rc = lib.orc_gmres(nb, mesh.ne, mesh.ned, _i(mesh.edges), _d(diag), _d(off), _d(inv), _d(b), _d(x),
                       m, ctypes.c_double(tol), max_it, _d(info))
    return x, int(info[0]), float(info[1]), rc == 0


def dense_solve(A, b):
    """Stiff\\F by dense LU with partial pivoting (Sec. 2.3)."""
    lib = _load()
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    x = np.array(b, dtype=np.float64, copy=True).reshape(-1)
    rc = lib.orc_dense_solve(A.shape[0], _d(A), _d(x))
    if rc != 0:
        raise ZeroDivisionError("singular matrix")
    return x


def dense_matrix(mesh: Mesh, diag, off):
    return to_sparse(mesh, diag, off).toarray()


def nonlinear(mesh: Mesh, k: int, coef, p: int, c: float):
    """The paper's nonlinear_global (Sec. 3): H(v) and HJ(v) of Eq. (newton)
    for r(u) = c u^p.  Returns H [ne*nb] and HJ [ne, nb, nb] (element-diagonal
    blocks of the Jacobian of H)."""
    lib = _load()
    nb = nbasis(k)
    coef = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    H = np.zeros(mesh.ne * nb)
    HJ = np.zeros((mesh.ne, nb, nb))
    lib.orc_nonlinear(k, _d(mesh.nodes), mesh.ne, _i(mesh.elems), _d(coef), int(p), ctypes.c_double(c),
                      _d(H), _d(HJ))
    return H, HJ


def newton(mesh: Mesh, system: System, p: int, c: float, tol: float = 1e-10, max_newton: int = 50):
    """Newton's method of Eq. (newton) for D v + C v + R v + H(v) = F:
    v^0 = 0; Res^k = A v^k + H(v^k) - F; J^k = A + HJ(v^k); J^k w^k = -Res^k
    (sparse LU); v^{k+1} = v^k + w^k.  Stops when ||Res^k|| <= tol ||F||
    (reading of the paper's test on the linear residual) or after max_newton
    corrections.  Returns (v, corrections, [||Res^0||/||F||, ...])."""
    import scipy.sparse.linalg as spla
    k = system.k
    A = to_sparse(mesh, system.A_diag, system.A_off)
    F = system.F
    nF = np.linalg.norm(F)
    v = np.zeros_like(F)
    hist = []
    for it in range(max_newton + 1):
        H, HJ = nonlinear(mesh, k, v, p, c)
        res = A @ v + H - F
        hist.append(np.linalg.norm(res) / nF)
        if hist[-1] <= tol or it == max_newton:
            return v, it, hist
        J = to_sparse(mesh, system.A_diag + HJ, system.A_off)
        v = v + spla.spsolve(J.tocsc(), -res)
    return v, max_newton, hist


def l2_error(mesh: Mesh, k: int, coef, uex_q):
    """The paper's dg_error (Sec. 2.4): (||u_h - u||_L2, h_max); uex_q at
    quad_points(ERROR)."""
    lib = _load()
    out = np.zeros(2)
    coef = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    uex_q = np.ascontiguousarray(uex_q, dtype=np.float64).reshape(-1)
    lib.orc_l2_error(k, _d(mesh.nodes), mesh.ne, _i(mesh.elems), _d(coef), _d(uex_q), _d(out))
    return float(out[0]), float(out[1])


def evaluate(mesh: Mesh, k: int, coef, elem_ids, xy, want_basis=False):
    """u_h at physical points xy[p] inside elements elem_ids[p]; optionally the
    oracle basis values there."""
    lib = _load()
    elem_ids = np.ascontiguousarray(elem_ids, dtype=np.int32).reshape(-1)
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    npnt = elem_ids.shape[0]
    u = np.zeros(npnt)
    phi = np.zeros((npnt, nbasis(k))) if want_basis else None
    c = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    lib.orc_eval(k, _d(mesh.nodes), _i(mesh.elems), _d(c), npnt, _i(elem_ids), _d(xy), _d(u), _d(phi))
    return (u, phi) if want_basis else u
