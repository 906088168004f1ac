/*
 * dg_oracle.c -- plain FP64 CPU oracle for the interior-penalty DG method of
 * Uzunca & Karasozen, "A Matlab Tutorial for Diffusion-Convection-Reaction
 * Equations using DGFEM" (arXiv:1502.02941).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes (all in double precision, with scalar loops that follow the
 * paper's definitions term by term):
 *   - the mesh skeleton: interior / Dirichlet / Neumann edges with K_i < K_j
 *     and n_e pointing from K_i to K_j (Sec. 1, jump/average definitions,
 *     Fig. 1; mesh arrays of Sec. 2.1);
 *   - uniform (red) refinement of a triangulation (Sec. 2.1);
 *   - the matrices D, C, R and the vector F of Eq. (dgscheme)/(system):
 *     D = diffusion + interior penalty terms, C = convection + upwind terms,
 *     R = linear reaction, F_i = l_h(phi_i);
 *   - y = (D+C+R) x, a block-Jacobi preconditioned restarted GMRES(m)
 *     (Saad & Schultz 1986, modified Gram-Schmidt Arnoldi, Givens rotations),
 *     a dense LU solve with partial pivoting (the "Stiff\F" of Sec. 2.3);
 *   - the L2 error and h_max reported by the paper's dg_error (Sec. 2.4);
 *   - the non-linear reaction vector H(v) and its Jacobian HJ(v) of Sec. 3
 *     (Eq. (nonlinsystem), (newton)) for r(u) = c u^p.
 *
 * Basis: scaled monomials ((x-xc)/hK)^a ((y-yc)/hK)^b, a+b <= k, on each
 * element (the paper's "Equation.base = 1" option, Sec. 4 set_parameter).
 *
 * Readings of the paper taken here (where it is silent, ambiguous or garbled):
 *   A-1  RHS Dirichlet consistency term is  +kappa*eps*grad(v).n*gD  (equal to
 *        the printed -eps*grad(v).n*gD for SIPG); flag `literal_rhs` restores
 *        the printed sign for every method.
 *   A-3  h_e = |e| (edge length), raised to the superpenalisation exponent b0
 *        of set_parameter (Sec. 4; the paper's default b0 = 1): the penalty
 *        terms carry sigma eps / |e|^b0.
 *   A-5  upwind decision taken pointwise at each edge quadrature point with the
 *        strict inequality b.n < 0 (weight min(b.n,0)).
 *   A-6  the inflow-boundary terms are applied on every boundary edge where
 *        b.n < 0, Dirichlet or Neumann, with g taken from the Dirichlet data
 *        array, which the caller fills on all boundary edges.
 *   A-8  quadrature: Gauss-Legendre with k+2 points on edges, Duffy-collapsed
 *        Gauss-Legendre (k+2)^2 on triangles, (k+4)^2 for the L2 error; nodes
 *        from Newton iteration on the Legendre three-term recurrence.
 *
 * Coefficients: eps and alpha constant, b affine
 *   b(x,y) = (b[0] + b[1] x + b[2] y,  b[3] + b[4] x + b[5] y);
 * f at the volume quadrature points, gD and gN at the boundary-edge
 * quadrature points, both in the point order returned by orc_quad_points.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/*
 * Timing build only: compiled with -DORC_OPENMP -fopenmp (liboracle_omp.so)
 * the element, edge and vector loops of the apply, the block-Jacobi apply
 * and GMRES run on all host cores (edge contributions added atomically, dot
 * products as OpenMP reductions, so the last bits of the rounding differ).
 * The build the tests use has no such pragmas: it is the plain serial code.
 */
#ifdef ORC_OPENMP
#include <omp.h>
#define ORC_PAR(x) _Pragma(x)
#else
#define ORC_PAR(x)
#endif

/* Threads the loops above run on (1 in the serial build). */
int orc_num_threads(void)
{
#ifdef ORC_OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_MAXK 4
#define ORC_MAXNB 15   /* (k+1)(k+2)/2 for k = 4 */
#define ORC_MAXQ 16    /* Gauss points per direction */

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] by Newton iteration on P_n.                  */
/* ------------------------------------------------------------------------ */
static void legendre_and_derivative(int n, double x, double* p, double* dp)
{
    /* three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1} */
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int j = 1; j < n; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1; p1 = p2;
    }
    *p = p1;
    /* P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1) */
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

void orc_gauss_legendre01(int n, double* t, double* w)
{
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_and_derivative(n, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p, dp;
        legendre_and_derivative(n, x, &p, &dp);
        /* map [-1,1] -> [0,1]: t = (1 - x)/2 gives increasing t */
        t[i] = 0.5 * (1.0 - x);
        w[i] = 1.0 / ((1.0 - x * x) * dp * dp); /* (2/((1-x^2)P'^2)) / 2 */
    }
}

/* Duffy-collapsed rule on the reference triangle (0,0),(1,0),(0,1):
   r = u (1 - v), s = v, weight = wu wv (1 - v).  n*n points, index a*n+b
   for u-node a and v-node b.  Weights sum to 1/2. */
static void duffy_rule(int n, double* r, double* s, double* w)
{
    double t[ORC_MAXQ], tw[ORC_MAXQ];
    orc_gauss_legendre01(n, t, tw);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            r[a * n + b] = t[a] * (1.0 - t[b]);
            s[a * n + b] = t[b];
            w[a * n + b] = tw[a] * tw[b] * (1.0 - t[b]);
        }
}

/* ------------------------------------------------------------------------ */
/* Mesh skeleton (Sec. 2.1 arrays -> edge table).                            */
/* ------------------------------------------------------------------------ */
typedef struct { int lo, hi, elem, face; } face_rec;

static int cmp_face(const void* a, const void* b)
{
    const face_rec* x = (const face_rec*)a; const face_rec* y = (const face_rec*)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->elem != y->elem) return x->elem < y->elem ? -1 : 1;
    return 0;
}

typedef struct { int lo, hi, type; } bc_rec;

static int cmp_bc(const void* a, const void* b)
{
    const bc_rec* x = (const bc_rec*)a; const bc_rec* y = (const bc_rec*)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return 0;
}

/*
 * Build the edge table.  Inputs are 0-based: nodes[nv][2], elems[ne][3]
 * (counter-clockwise), dir[nd][2], neu[nn][2] (start/end node of each
 * boundary edge).
 * Output edges[e][5] = {va, vb, Ki, Kj, type}: va->vb is the edge as
 * traversed counter-clockwise by Ki, so rot(vb-va) is the outward normal of Ki
 * (= n_e from K_i to K_j for interior edges, Fig. 1).  Interior edges have
 * Ki < Kj and type 0; boundary edges have Kj = -1 and type 1 (Dirichlet) or
 * 2 (Neumann).  elem_edges[K][f] = index of the edge v_f -> v_{f+1} of K.
 * Returns the number of edges, or a negative error code:
 *   -1 element not counter-clockwise, -2 edge shared by more than two
 *   elements, -3 boundary edge without a boundary condition, -4 bad index.
 */
int orc_edges(int nv, const double* nodes, int ne, const int* elems,
              int nd, const int* dir, int nn, const int* neu,
              int* edges, int* elem_edges)
{
    for (int K = 0; K < ne; ++K) {
        for (int f = 0; f < 3; ++f)
            if (elems[3 * K + f] < 0 || elems[3 * K + f] >= nv) return -4;
        const double* a = nodes + 2 * elems[3 * K + 0];
        const double* b = nodes + 2 * elems[3 * K + 1];
        const double* c = nodes + 2 * elems[3 * K + 2];
        double area2 = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
        if (!(area2 > 0.0)) return -1;
    }
    face_rec* fr = (face_rec*)malloc(sizeof(face_rec) * (size_t)(3 * ne));
    for (int K = 0; K < ne; ++K)
        for (int f = 0; f < 3; ++f) {
            int va = elems[3 * K + f], vb = elems[3 * K + (f + 1) % 3];
            face_rec r = { va < vb ? va : vb, va < vb ? vb : va, K, f };
            fr[3 * K + f] = r;
        }
    qsort(fr, (size_t)(3 * ne), sizeof(face_rec), cmp_face);

    int nbc = nd + nn;
    bc_rec* bc = (bc_rec*)malloc(sizeof(bc_rec) * (size_t)(nbc > 0 ? nbc : 1));
    for (int i = 0; i < nd; ++i) {
        int a = dir[2 * i], b = dir[2 * i + 1];
        bc_rec r = { a < b ? a : b, a < b ? b : a, 1 }; bc[i] = r;
    }
    for (int i = 0; i < nn; ++i) {
        int a = neu[2 * i], b = neu[2 * i + 1];
        bc_rec r = { a < b ? a : b, a < b ? b : a, 2 }; bc[nd + i] = r;
    }
    qsort(bc, (size_t)nbc, sizeof(bc_rec), cmp_bc);

    int ned = 0, err = 0;
    for (int i = 0; i < 3 * ne && !err;) {
        int j = i + 1;
        while (j < 3 * ne && fr[j].lo == fr[i].lo && fr[j].hi == fr[i].hi) ++j;
        int cnt = j - i;
        int* E = edges + 5 * ned;
        if (cnt == 2) {
            /* fr sorted by element: fr[i] is the lower element index K_i */
            const face_rec* Ki = &fr[i];
            E[0] = elems[3 * Ki->elem + Ki->face];
            E[1] = elems[3 * Ki->elem + (Ki->face + 1) % 3];
            E[2] = fr[i].elem; E[3] = fr[i + 1].elem; E[4] = 0;
            elem_edges[3 * fr[i].elem + fr[i].face] = ned;
            elem_edges[3 * fr[i + 1].elem + fr[i + 1].face] = ned;
        } else if (cnt == 1) {
            bc_rec key = { fr[i].lo, fr[i].hi, 0 };
            bc_rec* hit = (bc_rec*)bsearch(&key, bc, (size_t)nbc, sizeof(bc_rec), cmp_bc);
            if (!hit) { err = -3; break; }
            E[0] = elems[3 * fr[i].elem + fr[i].face];
            E[1] = elems[3 * fr[i].elem + (fr[i].face + 1) % 3];
            E[2] = fr[i].elem; E[3] = -1; E[4] = hit->type;
            elem_edges[3 * fr[i].elem + fr[i].face] = ned;
        } else {
            err = -2; break;
        }
        ++ned;
        i = j;
    }
    free(fr); free(bc);
    return err ? err : ned;
}

/*
 * Uniform red refinement (the paper's uniformrefine, Sec. 2.1): every edge is
 * split at its midpoint and every triangle (a,b,c) is replaced by
 * (a,m_ab,m_ca), (m_ab,b,m_bc), (m_ca,m_bc,c), (m_ab,m_bc,m_ca); boundary
 * edges are split into two with the same condition.  New nodes: the old ones,
 * then one midpoint per edge in edge order.  Outputs sized nv+ned, 4ne, 2nd,
 * 2nn.  Returns the number of new nodes or a negative orc_edges error.
 */
int orc_refine(int nv, const double* nodes, int ne, const int* elems,
               int nd, const int* dir, int nn, const int* neu,
               double* nodes_out, int* elems_out, int* dir_out, int* neu_out)
{
    int* edges = (int*)malloc(sizeof(int) * 5 * (size_t)(3 * ne));
    int* ee = (int*)malloc(sizeof(int) * 3 * (size_t)ne);
    int ned = orc_edges(nv, nodes, ne, elems, nd, dir, nn, neu, edges, ee);
    if (ned < 0) { free(edges); free(ee); return ned; }
    memcpy(nodes_out, nodes, sizeof(double) * 2 * (size_t)nv);
    for (int e = 0; e < ned; ++e) {
        const double* a = nodes + 2 * edges[5 * e];
        const double* b = nodes + 2 * edges[5 * e + 1];
        nodes_out[2 * (nv + e)] = 0.5 * (a[0] + b[0]);
        nodes_out[2 * (nv + e) + 1] = 0.5 * (a[1] + b[1]);
    }
    for (int K = 0; K < ne; ++K) {
        int a = elems[3 * K], b = elems[3 * K + 1], c = elems[3 * K + 2];
        int mab = nv + ee[3 * K + 0], mbc = nv + ee[3 * K + 1], mca = nv + ee[3 * K + 2];
        int* o = elems_out + 12 * K;
        o[0] = a;   o[1] = mab; o[2] = mca;
        o[3] = mab; o[4] = b;   o[5] = mbc;
        o[6] = mca; o[7] = mbc; o[8] = c;
        o[9] = mab; o[10] = mbc; o[11] = mca;
    }
    /* boundary lists: find the midpoint of each listed edge */
    for (int pass = 0; pass < 2; ++pass) {
        int n = pass == 0 ? nd : nn;
        const int* in = pass == 0 ? dir : neu;
        int* out = pass == 0 ? dir_out : neu_out;
        for (int i = 0; i < n; ++i) {
            int a = in[2 * i], b = in[2 * i + 1], m = -1;
            for (int e = 0; e < ned; ++e)
                if (edges[5 * e + 3] < 0 &&
                    ((edges[5 * e] == a && edges[5 * e + 1] == b) ||
                     (edges[5 * e] == b && edges[5 * e + 1] == a))) { m = nv + e; break; }
            if (m < 0) { free(edges); free(ee); return -3; }
            out[4 * i] = a; out[4 * i + 1] = m; out[4 * i + 2] = m; out[4 * i + 3] = b;
        }
    }
    free(edges); free(ee);
    return nv + ned;
}

/* ------------------------------------------------------------------------ */
/* Element geometry and scaled-monomial basis.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double v[3][2];   /* vertices */
    double xc, yc;    /* centroid */
    double hK;        /* diameter = longest edge */
    double area;
} elem_geo;

static void element_geometry(const double* nodes, const int* elems, int K, elem_geo* g)
{
    for (int i = 0; i < 3; ++i) {
        g->v[i][0] = nodes[2 * elems[3 * K + i]];
        g->v[i][1] = nodes[2 * elems[3 * K + i] + 1];
    }
    g->xc = (g->v[0][0] + g->v[1][0] + g->v[2][0]) / 3.0;
    g->yc = (g->v[0][1] + g->v[1][1] + g->v[2][1]) / 3.0;
    g->hK = 0.0;
    for (int i = 0; i < 3; ++i) {
        double dx = g->v[(i + 1) % 3][0] - g->v[i][0];
        double dy = g->v[(i + 1) % 3][1] - g->v[i][1];
        double l = sqrt(dx * dx + dy * dy);
        if (l > g->hK) g->hK = l;
    }
    g->area = 0.5 * ((g->v[1][0] - g->v[0][0]) * (g->v[2][1] - g->v[0][1]) -
                     (g->v[1][1] - g->v[0][1]) * (g->v[2][0] - g->v[0][0]));
}

/* physical point of reference coordinates (r,s) */
static void ref_to_phys(const elem_geo* g, double r, double s, double* x, double* y)
{
    *x = g->v[0][0] + r * (g->v[1][0] - g->v[0][0]) + s * (g->v[2][0] - g->v[0][0]);
    *y = g->v[0][1] + r * (g->v[1][1] - g->v[0][1]) + s * (g->v[2][1] - g->v[0][1]);
}

static int nbasis(int k) { return (k + 1) * (k + 2) / 2; }

static double ipow(double x, int n) { double r = 1.0; for (int i = 0; i < n; ++i) r *= x; return r; }

/* phi_m, m over (a,b) with a+b = d for d = 0..k, a from d down to 0 */
static void monomial_basis(const elem_geo* g, int k, double x, double y,
                           double* phi, double* dphix, double* dphiy)
{
    double X = (x - g->xc) / g->hK, Y = (y - g->yc) / g->hK;
    int m = 0;
    for (int d = 0; d <= k; ++d)
        for (int a = d; a >= 0; --a) {
            int b = d - a;
            phi[m] = ipow(X, a) * ipow(Y, b);
            dphix[m] = a > 0 ? a * ipow(X, a - 1) * ipow(Y, b) / g->hK : 0.0;
            dphiy[m] = b > 0 ? b * ipow(X, a) * ipow(Y, b - 1) / g->hK : 0.0;
            ++m;
        }
}

/* ------------------------------------------------------------------------ */
/* Quadrature points in physical coordinates.                                */
/* ------------------------------------------------------------------------ */
/*
 * which = 0: volume points, [ne][(k+2)^2][2]
 * which = 1: boundary-edge points, [n boundary edges, in edge order][k+2][2],
 *            each edge traversed from va to vb (counter-clockwise for Ki)
 * which = 2: L2-error points, [ne][(k+4)^2][2]
 * which = 3: points of every edge, [ned][k+2][2], in edge order, each edge
 *            traversed from va to vb (where a variable eps is evaluated)
 */
void orc_quad_points(int which, int k, const double* nodes, int ne, const int* elems,
                     int ned, const int* edges, double* out)
{
    if (which == 0 || which == 2) {
        int n = which == 0 ? k + 2 : k + 4;
        double r[ORC_MAXQ * ORC_MAXQ], s[ORC_MAXQ * ORC_MAXQ], w[ORC_MAXQ * ORC_MAXQ];
        duffy_rule(n, r, s, w);
        for (int K = 0; K < ne; ++K) {
            elem_geo g; element_geometry(nodes, elems, K, &g);
            for (int q = 0; q < n * n; ++q)
                ref_to_phys(&g, r[q], s[q], &out[2 * ((size_t)K * n * n + q)],
                            &out[2 * ((size_t)K * n * n + q) + 1]);
        }
    } else {
        int n = k + 2;
        double t[ORC_MAXQ], tw[ORC_MAXQ];
        orc_gauss_legendre01(n, t, tw);
        size_t ib = 0;
        for (int e = 0; e < ned; ++e) {
            if (which == 1 && edges[5 * e + 3] >= 0) continue;
            const double* a = nodes + 2 * edges[5 * e];
            const double* b = nodes + 2 * edges[5 * e + 1];
            for (int q = 0; q < n; ++q) {
                out[2 * (ib * n + q)] = a[0] + t[q] * (b[0] - a[0]);
                out[2 * (ib * n + q) + 1] = a[1] + t[q] * (b[1] - a[1]);
            }
            ++ib;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Assembly of D, C, R and F (Eq. (dgscheme) and (system)).                  */
/* ------------------------------------------------------------------------ */
/*
 * Block storage shared by the oracle routines below:
 *   diag[K][i][j]          block (K,K):   row = test phi_i on K, col = trial phi_j on K
 *   off[e][0][i][j]        block (Ki,Kj): row on Ki, col on Kj (interior edge e)
 *   off[e][1][i][j]        block (Kj,Ki): row on Kj, col on Ki
 * Entry = form(phi_j, phi_i) as in Eq. (system).  off[] has an entry for every
 * edge; boundary edges leave theirs zero.
 */
typedef struct {
    double kappa, sigma_int, sigma_bdry, eps, alpha;
    double b[6];
    int literal_rhs;
    double b0;        /* superpenalisation exponent: penalty sigma eps / |e|^b0 */
} orc_coeffs;

static void advection(const orc_coeffs* c, double x, double y, double* bx, double* by)
{
    *bx = c->b[0] + c->b[1] * x + c->b[2] * y;
    *by = c->b[3] + c->b[4] * x + c->b[5] * y;
}

#define BLK(p, idx, nb) ((p) + (size_t)(idx) * (nb) * (nb))

/*
 * Assemble.  D, C, R each have diag [ne*nb*nb] and off [ned*2*nb*nb] arrays
 * (zeroed here); pass C_* or R_* equal to D_* to accumulate into one matrix.
 * f_q: [ne][(k+2)^2] at the volume points; gD_q, gN_q: [nbe][k+2] at the
 * boundary-edge points (orc_quad_points order).  F: [ne][nb].
 * Diffusion: the constant eps, or, when eps_vol is given, the values of the
 * paper's fdiff(x, y) (Sec. 2.2) at the quadrature points: eps_vol
 * [ne][(k+2)^2] at the volume points (orc_quad_points 0) for the volume term,
 * eps_edge [ned][k+2] at the edge points (orc_quad_points 3) for the face
 * terms {eps grad u}, {eps grad v}, the penalty sigma eps / h_e and the RHS
 * Dirichlet terms (reading A-4: eps taken pointwise at each quadrature point).
 */
void orc_assemble(int k, const double* nodes, int ne, const int* elems,
                  int ned, const int* edges, const int* elem_edges,
                  double kappa, double sigma_int, double sigma_bdry,
                  double eps, double alpha, const double* b_affine, int literal_rhs, double b0,
                  const double* f_q, const double* gD_q, const double* gN_q,
                  const double* eps_vol, const double* eps_edge,
                  double* D_diag, double* D_off, double* C_diag, double* C_off,
                  double* R_diag, double* R_off, double* F)
{
    orc_coeffs cf;
    cf.kappa = kappa; cf.sigma_int = sigma_int; cf.sigma_bdry = sigma_bdry;
    cf.eps = eps; cf.alpha = alpha; cf.literal_rhs = literal_rhs; cf.b0 = b0;
    for (int i = 0; i < 6; ++i) cf.b[i] = b_affine[i];
    const int nb = nbasis(k);
    const size_t nb2 = (size_t)nb * nb;
    memset(D_diag, 0, sizeof(double) * ne * nb2);
    memset(D_off, 0, sizeof(double) * 2 * ned * nb2);
    if (C_diag != D_diag) { memset(C_diag, 0, sizeof(double) * ne * nb2); memset(C_off, 0, sizeof(double) * 2 * ned * nb2); }
    if (R_diag != D_diag && R_diag != C_diag) { memset(R_diag, 0, sizeof(double) * ne * nb2); memset(R_off, 0, sizeof(double) * 2 * ned * nb2); }
    memset(F, 0, sizeof(double) * ne * nb);
    (void)elem_edges;

    double phi[ORC_MAXNB], px[ORC_MAXNB], py[ORC_MAXNB];

    /* ---- element (volume) integrals ---------------------------------- */
    {
        int n = k + 2;
        double r[ORC_MAXQ * ORC_MAXQ], s[ORC_MAXQ * ORC_MAXQ], w[ORC_MAXQ * ORC_MAXQ];
        duffy_rule(n, r, s, w);
        for (int K = 0; K < ne; ++K) {
            elem_geo g; element_geometry(nodes, elems, K, &g);
            double detJ = 2.0 * g.area;
            for (int q = 0; q < n * n; ++q) {
                double x, y; ref_to_phys(&g, r[q], s[q], &x, &y);
                double wq = w[q] * detJ;
                double bx, by; advection(&cf, x, y, &bx, &by);
                monomial_basis(&g, k, x, y, phi, px, py);
                double fval = f_q[(size_t)K * n * n + q];
                double epsq = eps_vol ? eps_vol[(size_t)K * n * n + q] : cf.eps;
                for (int i = 0; i < nb; ++i) {          /* test  v = phi_i */
                    for (int j = 0; j < nb; ++j) {      /* trial u = phi_j */
                        /* D: eps grad u . grad v */
                        BLK(D_diag, K, nb)[i * nb + j] += wq * epsq * (px[j] * px[i] + py[j] * py[i]);
                        /* C: (b . grad u) v */
                        BLK(C_diag, K, nb)[i * nb + j] += wq * (bx * px[j] + by * py[j]) * phi[i];
                        /* R: alpha u v */
                        BLK(R_diag, K, nb)[i * nb + j] += wq * cf.alpha * phi[j] * phi[i];
                    }
                    F[K * nb + i] += wq * fval * phi[i];
                }
            }
        }
    }

    /* ---- edge integrals over Gamma_0 u Gamma_D (diffusion, penalty) ----- */
    int nq = k + 2;
    double t[ORC_MAXQ], tw[ORC_MAXQ];
    orc_gauss_legendre01(nq, t, tw);
    {
        size_t ib = 0;
        for (int e = 0; e < ned; ++e) {
            const int* E = edges + 5 * e;
            const double* a = nodes + 2 * E[0];
            const double* bpt = nodes + 2 * E[1];
            double dx = bpt[0] - a[0], dy = bpt[1] - a[1];
            double len = sqrt(dx * dx + dy * dy);
            double ne_x = dy / len, ne_y = -dx / len;   /* n_e: outward of Ki */
            double he = pow(len, cf.b0);                  /* A-3: h_e = |e|, raised to b0 */
            int type = E[4];
            int bidx = -1;
            if (E[3] < 0) bidx = (int)(ib++);
            if (type == 2) continue;                      /* Neumann: no IP terms */
            elem_geo gi, gj;
            element_geometry(nodes, elems, E[2], &gi);
            if (type == 0) element_geometry(nodes, elems, E[3], &gj);
            double sigma = type == 0 ? cf.sigma_int : cf.sigma_bdry;
            for (int q = 0; q < nq; ++q) {
                double x = a[0] + t[q] * dx, y = a[1] + t[q] * dy;
                double wq = tw[q] * len;
                double epsq = eps_vol ? eps_edge[(size_t)e * nq + q] : cf.eps;
                double phi_i[ORC_MAXNB], pxi[ORC_MAXNB], pyi[ORC_MAXNB];
                double phi_j[ORC_MAXNB], pxj[ORC_MAXNB], pyj[ORC_MAXNB];
                monomial_basis(&gi, k, x, y, phi_i, pxi, pyi);
                if (type == 0) monomial_basis(&gj, k, x, y, phi_j, pxj, pyj);
                /* sides: 0 = K_i, 1 = K_j.  For a basis function living on side
                   s, its traces are (value on Ki, value on Kj) with the other
                   side zero.  Jump [v] = (v_i - v_j) n_e, average {v} =
                   (v_i + v_j)/2 on interior edges; on Dirichlet edges [v] =
                   v_i n, {v} = v_i. */
                int nsides = type == 0 ? 2 : 1;
                for (int sv = 0; sv < nsides; ++sv)          /* side of test fn */
                    for (int su = 0; su < nsides; ++su) {    /* side of trial fn */
                        double* blk;
                        if (sv == 0 && su == 0) blk = BLK(D_diag, E[2], nb);
                        else if (sv == 1 && su == 1) blk = BLK(D_diag, E[3], nb);
                        else if (sv == 0 && su == 1) blk = BLK(D_off, 2 * e + 0, nb);
                        else blk = BLK(D_off, 2 * e + 1, nb);
                        const double* pv = sv == 0 ? phi_i : phi_j;
                        const double* pvx = sv == 0 ? pxi : pxj;
                        const double* pvy = sv == 0 ? pyi : pyj;
                        const double* pu = su == 0 ? phi_i : phi_j;
                        const double* pux = su == 0 ? pxi : pxj;
                        const double* puy = su == 0 ? pyi : pyj;
                        double sgn_v = sv == 0 ? 1.0 : -1.0;   /* v_i n_e - v_j n_e */
                        double sgn_u = su == 0 ? 1.0 : -1.0;
                        double avgw = type == 0 ? 0.5 : 1.0;
                        for (int i = 0; i < nb; ++i)
                            for (int j = 0; j < nb; ++j) {
                                /* [v] (vector) and {eps grad v}, {eps grad u} */
                                double jv_x = sgn_v * pv[i] * ne_x, jv_y = sgn_v * pv[i] * ne_y;
                                double ju_x = sgn_u * pu[j] * ne_x, ju_y = sgn_u * pu[j] * ne_y;
                                double agv_x = avgw * epsq * pvx[i], agv_y = avgw * epsq * pvy[i];
                                double agu_x = avgw * epsq * pux[j], agu_y = avgw * epsq * puy[j];
                                double val = -(agu_x * jv_x + agu_y * jv_y)
                                             + cf.kappa * (agv_x * ju_x + agv_y * ju_y)
                                             + sigma * epsq / he * (ju_x * jv_x + ju_y * jv_y);
                                blk[i * nb + j] += wq * val;
                            }
                    }
                if (type == 1) {
                    /* RHS Dirichlet term: gD (sigma eps/h_e v - eps grad v . n) as
                       printed, or with +kappa (reading A-1). */
                    double g = gD_q[(size_t)bidx * nq + q];
                    double cons = cf.literal_rhs ? -1.0 : cf.kappa;
                    for (int i = 0; i < nb; ++i)
                        F[E[2] * nb + i] += wq * g * (sigma * epsq / he * phi_i[i]
                                          + cons * epsq * (pxi[i] * ne_x + pyi[i] * ne_y));
                }
            }
        }
    }

    /* ---- upwind convection terms, element by element over dK^- ----------- */
    /* For boundary-edge data lookup: boundary index of each edge. */
    int* bindex = (int*)malloc(sizeof(int) * (size_t)(ned > 0 ? ned : 1));
    {
        int ib = 0;
        for (int e = 0; e < ned; ++e) bindex[e] = edges[5 * e + 3] < 0 ? ib++ : -1;
    }
    for (int K = 0; K < ne; ++K) {
        elem_geo g; element_geometry(nodes, elems, K, &g);
        for (int f = 0; f < 3; ++f) {
            int e = elem_edges[3 * K + f];
            const int* E = edges + 5 * e;
            /* this element's own traversal of the face: v_f -> v_{f+1} */
            const double* a = nodes + 2 * elems[3 * K + f];
            const double* bpt = nodes + 2 * elems[3 * K + (f + 1) % 3];
            double dx = bpt[0] - a[0], dy = bpt[1] - a[1];
            double len = sqrt(dx * dx + dy * dy);
            double nx = dy / len, ny = -dx / len;         /* n_K outward */
            int other = E[3] < 0 ? -1 : (E[2] == K ? E[3] : E[2]);
            elem_geo go;
            if (other >= 0) element_geometry(nodes, elems, other, &go);
            for (int q = 0; q < nq; ++q) {
                double x = a[0] + t[q] * dx, y = a[1] + t[q] * dy;
                double wq = tw[q] * len;
                double bx, by; advection(&cf, x, y, &bx, &by);
                double bn = bx * nx + by * ny;
                if (!(bn < 0.0)) continue;                  /* x not in dK^- */
                double pin[ORC_MAXNB], dxi[ORC_MAXNB], dyi[ORC_MAXNB];
                monomial_basis(&g, k, x, y, pin, dxi, dyi);
                if (other >= 0) {
                    /* + b.n (u_out - u_in) v */
                    double pout[ORC_MAXNB], dxo[ORC_MAXNB], dyo[ORC_MAXNB];
                    monomial_basis(&go, k, x, y, pout, dxo, dyo);
                    double* blk_out = (E[2] == K) ? BLK(C_off, 2 * e + 0, nb) : BLK(C_off, 2 * e + 1, nb);
                    for (int i = 0; i < nb; ++i)
                        for (int j = 0; j < nb; ++j) {
                            blk_out[i * nb + j] += wq * bn * pout[j] * pin[i];
                            BLK(C_diag, K, nb)[i * nb + j] -= wq * bn * pin[j] * pin[i];
                        }
                } else {
                    /* x in dK^- n Gamma^-:  - b.n u_in v  and RHS  - b.n gD v.
                       The boundary point sequence of edge e runs va -> vb, which
                       is this element's own traversal, so q indexes it directly. */
                    double g = gD_q[(size_t)bindex[e] * nq + q];
                    for (int i = 0; i < nb; ++i) {
                        for (int j = 0; j < nb; ++j)
                            BLK(C_diag, K, nb)[i * nb + j] -= wq * bn * pin[j] * pin[i];
                        F[K * nb + i] -= wq * bn * g * pin[i];
                    }
                }
            }
        }
    }

    /* ---- Neumann data ----------------------------------------------------- */
    for (int e = 0; e < ned; ++e) {
        const int* E = edges + 5 * e;
        if (E[4] != 2) continue;
        elem_geo g; element_geometry(nodes, elems, E[2], &g);
        const double* a = nodes + 2 * E[0];
        const double* bpt = nodes + 2 * E[1];
        double dx = bpt[0] - a[0], dy = bpt[1] - a[1];
        double len = sqrt(dx * dx + dy * dy);
        for (int q = 0; q < nq; ++q) {
            double x = a[0] + t[q] * dx, y = a[1] + t[q] * dy;
            double pin[ORC_MAXNB], d1[ORC_MAXNB], d2[ORC_MAXNB];
            monomial_basis(&g, k, x, y, pin, d1, d2);
            double gn = gN_q[(size_t)bindex[e] * nq + q];
            for (int i = 0; i < nb; ++i) F[E[2] * nb + i] += tw[q] * len * gn * pin[i];
        }
    }
    free(bindex);
}

/* ------------------------------------------------------------------------ */
/* y = A x with the block storage above.                                     */
/* ------------------------------------------------------------------------ */
void orc_apply(int nb, int ne, int ned, const int* edges,
               const double* diag, const double* off, const double* x, double* y)
{
    ORC_PAR("omp parallel for schedule(static)")
    for (int K = 0; K < ne; ++K)
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < nb; ++j) s += BLK(diag, K, nb)[i * nb + j] * x[K * nb + j];
            y[K * nb + i] = s;
        }
    ORC_PAR("omp parallel for schedule(static)")
    for (int e = 0; e < ned; ++e) {
        int Ki = edges[5 * e + 2], Kj = edges[5 * e + 3];
        if (Kj < 0) continue;
        for (int i = 0; i < nb; ++i) {
            double s0 = 0.0, s1 = 0.0;
            for (int j = 0; j < nb; ++j) {
                s0 += BLK(off, 2 * e + 0, nb)[i * nb + j] * x[Kj * nb + j];
                s1 += BLK(off, 2 * e + 1, nb)[i * nb + j] * x[Ki * nb + j];
            }
            ORC_PAR("omp atomic")
            y[Ki * nb + i] += s0;
            ORC_PAR("omp atomic")
            y[Kj * nb + i] += s1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (Stiff\F), and small-block inverses.       */
/* ------------------------------------------------------------------------ */
/* Solves A x = b in place: A [n][n] row-major is overwritten by its LU
   factors, b by x.  Returns 0, or -1 if a zero pivot is met. */
int orc_dense_solve(int n, double* A, double* b)
{
    int* piv = (int*)malloc(sizeof(int) * (size_t)n);
    for (int c = 0; c < n; ++c) {
        int p = c; double best = fabs(A[(size_t)c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + c]) > best) { best = fabs(A[(size_t)r * n + c]); p = r; }
        if (best == 0.0) { free(piv); return -1; }
        piv[c] = p;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                double tmp = A[(size_t)c * n + j]; A[(size_t)c * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = tmp;
            }
            double tmp = b[c]; b[c] = b[p]; b[p] = tmp;
        }
        for (int r = c + 1; r < n; ++r) {
            double l = A[(size_t)r * n + c] / A[(size_t)c * n + c];
            A[(size_t)r * n + c] = l;
            for (int j = c + 1; j < n; ++j) A[(size_t)r * n + j] -= l * A[(size_t)c * n + j];
            b[r] -= l * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[(size_t)r * n + j] * b[j];
        b[r] = s / A[(size_t)r * n + r];
    }
    free(piv);
    return 0;
}

/* Gauss-Jordan inverse with partial pivoting of an nb x nb block. */
static int block_inverse(int nb, const double* A, double* Ainv)
{
    double M[ORC_MAXNB][2 * ORC_MAXNB];
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < 2 * nb; ++j)
            M[i][j] = j < nb ? A[i * nb + j] : (j - nb == i ? 1.0 : 0.0);
    for (int c = 0; c < nb; ++c) {
        int p = c;
        for (int r = c + 1; r < nb; ++r) if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (M[p][c] == 0.0) return -1;
        if (p != c) for (int j = 0; j < 2 * nb; ++j) { double tmp = M[c][j]; M[c][j] = M[p][j]; M[p][j] = tmp; }
        double d = M[c][c];
        for (int j = 0; j < 2 * nb; ++j) M[c][j] /= d;
        for (int r = 0; r < nb; ++r) {
            if (r == c) continue;
            double l = M[r][c];
            if (l != 0.0) for (int j = 0; j < 2 * nb; ++j) M[r][j] -= l * M[c][j];
        }
    }
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) Ainv[i * nb + j] = M[i][nb + j];
    return 0;
}

/* Inverses of all diagonal blocks; returns 0 or -(1+K) for a singular block. */
int orc_block_jacobi(int nb, int ne, const double* diag, double* inv)
{
    for (int K = 0; K < ne; ++K)
        if (block_inverse(nb, BLK(diag, K, nb), BLK(inv, K, nb)) != 0) return -(1 + K);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(m), right block-Jacobi preconditioning, x0 = 0.           */
/* ------------------------------------------------------------------------ */
static double dotv(size_t n, const double* a, const double* b)
{
    double s = 0.0;
    ORC_PAR("omp parallel for reduction(+:s) schedule(static)")
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void bj_apply(int nb, int ne, const double* inv, const double* r, double* z)
{
    ORC_PAR("omp parallel for schedule(static)")
    for (int K = 0; K < ne; ++K)
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < nb; ++j) s += BLK(inv, K, nb)[i * nb + j] * r[K * nb + j];
            z[K * nb + i] = s;
        }
}

/*
 * Solves (diag,off) x = b.  inv = block-Jacobi inverses (orc_block_jacobi),
 * or NULL for no preconditioner.  Stops when ||b - A x||_2 <= tol ||b||_2
 * (true residual, checked at each restart and at the end) or after max_it
 * Arnoldi steps.  info[0] = iterations, info[1] = final relative residual.
 * Returns 0 when converged, 1 otherwise.
 */
int orc_gmres(int nb, int ne, int ned, const int* edges, const double* diag, const double* off,
              const double* inv, const double* b, double* x, int m, double tol, int max_it,
              double* info)
{
    size_t n = (size_t)ne * nb;
    double* V = (double*)malloc(sizeof(double) * n * (size_t)(m + 1));
    double* w = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * m);
    double* sn = (double*)malloc(sizeof(double) * m);
    double* gvec = (double*)malloc(sizeof(double) * (m + 1));
    double* yv = (double*)malloc(sizeof(double) * m);
    memset(x, 0, sizeof(double) * n);
    double bnorm = sqrt(dotv(n, b, b));
    int its = 0, converged = 0;
    double relres = 1.0;
    if (bnorm == 0.0) { info[0] = 0; info[1] = 0.0; converged = 1; goto done; }
    for (;;) {
        /* r = b - A x */
        orc_apply(nb, ne, ned, edges, diag, off, x, w);
        ORC_PAR("omp parallel for schedule(static)")
        for (size_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
        double beta = sqrt(dotv(n, w, w));
        relres = beta / bnorm;
        if (relres <= tol) { converged = 1; break; }
        if (its >= max_it) break;
        ORC_PAR("omp parallel for schedule(static)")
        for (size_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(gvec, 0, sizeof(double) * (m + 1));
        gvec[0] = beta;
        int j;
        for (j = 0; j < m && its < max_it; ++j) {
            ++its;
            double* vj = V + (size_t)j * n;
            if (inv) bj_apply(nb, ne, inv, vj, z); else memcpy(z, vj, sizeof(double) * n);
            orc_apply(nb, ne, ned, edges, diag, off, z, w);
            for (int i = 0; i <= j; ++i) {                     /* modified Gram-Schmidt */
                double h = dotv(n, w, V + (size_t)i * n);
                H[i * m + j] = h;
                ORC_PAR("omp parallel for schedule(static)")
                for (size_t l = 0; l < n; ++l) w[l] -= h * V[(size_t)i * n + l];
            }
            double hn = sqrt(dotv(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0) {
                ORC_PAR("omp parallel for schedule(static)")
                for (size_t l = 0; l < n; ++l) V[(size_t)(j + 1) * n + l] = w[l] / hn;
            }
            for (int i = 0; i < j; ++i) {                      /* previous rotations */
                double t1 = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                double t2 = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t1; H[(i + 1) * m + j] = t2;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double r = sqrt(a * a + bb * bb);
            cs[j] = r == 0.0 ? 1.0 : a / r; sn[j] = r == 0.0 ? 0.0 : bb / r;
            H[j * m + j] = r; H[(j + 1) * m + j] = 0.0;
            gvec[j + 1] = -sn[j] * gvec[j]; gvec[j] = cs[j] * gvec[j];
            if (fabs(gvec[j + 1]) <= tol * bnorm || hn == 0.0) { ++j; break; }
        }
        /* solve the j x j triangular system and update x += M^-1 V y */
        for (int i = j - 1; i >= 0; --i) {
            double s = gvec[i];
            for (int l = i + 1; l < j; ++l) s -= H[i * m + l] * yv[l];
            yv[i] = s / H[i * m + i];
        }
        memset(w, 0, sizeof(double) * n);
        for (int i = 0; i < j; ++i) {
            ORC_PAR("omp parallel for schedule(static)")
            for (size_t l = 0; l < n; ++l) w[l] += yv[i] * V[(size_t)i * n + l];
        }
        if (inv) bj_apply(nb, ne, inv, w, z); else memcpy(z, w, sizeof(double) * n);
        ORC_PAR("omp parallel for schedule(static)")
        for (size_t l = 0; l < n; ++l) x[l] += z[l];
    }
    info[0] = its; info[1] = relres;
done:
    free(V); free(w); free(z); free(H); free(cs); free(sn); free(gvec); free(yv);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Non-linear reaction (Sec. 3, Eq. (nonlin)): the vector H and its Jacobian  */
/* HJ of Eq. (nonlinsystem)/(newton) for r(u) = c u^p,                       */
/*   H_i(v)  = int_K r(u_h) phi_i,     u_h = sum_j v_j phi_j on K,           */
/*   HJ_ij(v) = dH_i/dv_j = int_K r'(u_h) phi_j phi_i   (element-diagonal),  */
/* with the volume rule of the assembly ((k+2)^2 Duffy points).             */
/* H [ne*nb], HJ [ne][nb][nb] (row i = test function, column j = trial).    */
/* ------------------------------------------------------------------------ */
void orc_nonlinear(int k, const double* nodes, int ne, const int* elems, const double* coef,
                   int p, double c, double* H, double* HJ)
{
    int n = k + 2, nb = nbasis(k);
    double r[ORC_MAXQ * ORC_MAXQ], s[ORC_MAXQ * ORC_MAXQ], w[ORC_MAXQ * ORC_MAXQ];
    duffy_rule(n, r, s, w);
    double phi[ORC_MAXNB], d1[ORC_MAXNB], d2[ORC_MAXNB];
    memset(H, 0, sizeof(double) * (size_t)ne * nb);
    memset(HJ, 0, sizeof(double) * (size_t)ne * nb * nb);
    for (int K = 0; K < ne; ++K) {
        elem_geo g; element_geometry(nodes, elems, K, &g);
        double detJ = 2.0 * g.area;
        for (int q = 0; q < n * n; ++q) {
            double x, y; ref_to_phys(&g, r[q], s[q], &x, &y);
            monomial_basis(&g, k, x, y, phi, d1, d2);
            double uh = 0.0;
            for (int j = 0; j < nb; ++j) uh += coef[(size_t)K * nb + j] * phi[j];
            double rv = c * ipow(uh, p);                       /* r(u_h)  */
            double dr = p >= 1 ? c * p * ipow(uh, p - 1) : 0.0; /* r'(u_h) */
            double wq = w[q] * detJ;
            for (int i = 0; i < nb; ++i) {
                H[(size_t)K * nb + i] += wq * rv * phi[i];
                for (int j = 0; j < nb; ++j)
                    HJ[((size_t)K * nb + i) * nb + j] += wq * dr * phi[j] * phi[i];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Post-processing (the paper's dg_error): L2 error, h_max; point values.    */
/* ------------------------------------------------------------------------ */
/* uex_q at the L2-error points (orc_quad_points which = 2).
   out[0] = ||u_h - u||_L2, out[1] = h_max (longest edge of the mesh). */
void orc_l2_error(int k, const double* nodes, int ne, const int* elems,
                  const double* coef, const double* uex_q, double* out)
{
    int n = k + 4, nb = nbasis(k);
    double r[ORC_MAXQ * ORC_MAXQ], s[ORC_MAXQ * ORC_MAXQ], w[ORC_MAXQ * ORC_MAXQ];
    duffy_rule(n, r, s, w);
    double err2 = 0.0, hmax = 0.0;
    double phi[ORC_MAXNB], d1[ORC_MAXNB], d2[ORC_MAXNB];
    for (int K = 0; K < ne; ++K) {
        elem_geo g; element_geometry(nodes, elems, K, &g);
        if (g.hK > hmax) hmax = g.hK;
        for (int q = 0; q < n * n; ++q) {
            double x, y; ref_to_phys(&g, r[q], s[q], &x, &y);
            monomial_basis(&g, k, x, y, phi, d1, d2);
            double uh = 0.0;
            for (int i = 0; i < nb; ++i) uh += coef[K * nb + i] * phi[i];
            double d = uh - uex_q[(size_t)K * n * n + q];
            err2 += w[q] * 2.0 * g.area * d * d;
        }
    }
    out[0] = sqrt(err2);
    out[1] = hmax;
}

/* u_h(x_p, y_p) on element elem[p] for np points; optionally the basis values
   phi_out[np][nb] (for change-of-basis tests). */
void orc_eval(int k, const double* nodes, const int* elems, const double* coef,
              int np, const int* elem, const double* xy, double* u_out, double* phi_out)
{
    int nb = nbasis(k);
    double phi[ORC_MAXNB], d1[ORC_MAXNB], d2[ORC_MAXNB];
    for (int p = 0; p < np; ++p) {
        elem_geo g; element_geometry(nodes, elems, elem[p], &g);
        monomial_basis(&g, k, xy[2 * p], xy[2 * p + 1], phi, d1, d2);
        double u = 0.0;
        for (int i = 0; i < nb; ++i) {
            if (coef) u += coef[elem[p] * nb + i] * phi[i];
            if (phi_out) phi_out[(size_t)p * nb + i] = phi[i];
        }
        if (u_out) u_out[p] = u;
    }
}
