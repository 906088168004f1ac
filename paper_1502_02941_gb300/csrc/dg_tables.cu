// dg_tables.cu -- reference-element data: quadrature rules and the
// orthonormal Dubiner basis with its gradients at the quadrature points.
// Built once per degree on the host in f64 and uploaded; the assembly, RHS,
// L2-error and evaluation kernels stage these tables in shared memory.
//
// Quadrature (the paper does not fix one): Gauss-Legendre with k+2 nodes on
// edges, the Duffy-collapsed tensor rule with (k+2)^2 nodes on the triangle
// (exact for total degree 2k+2, i.e. for every element integrand with affine b),
// and (k+4)^2 nodes for the L2 error.
#include <math.h>
#include <string.h>

#include <vector>

#include "dg_internal.cuh"

// Gauss-Legendre nodes/weights on [0,1], increasing nodes.  Each root of P_n
// is polished by Newton's method from the asymptotic guess; P_n and P_n' come
// from the three-term recurrence.
void dg_gauss_legendre01(int n, double* t, double* w) {
    for (int i = 0; i < n; ++i) {
        // i-th root counted from x = -1
        double x = -cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0.0, dpn = 1.0;
        for (int it = 0; it < 60; ++it) {
            double pm1 = 1.0, p = x;
            for (int j = 2; j <= n; ++j) {
                double pj = ((2 * j - 1) * x * p - (j - 1) * pm1) / j;
                pm1 = p;
                p = pj;
            }
            if (n == 1) { p = x; pm1 = 1.0; }
            pn = p;
            dpn = n * (pm1 - x * p) / (1.0 - x * x);
            double step = pn / dpn;
            x -= step;
            if (fabs(step) <= 1e-17) break;
        }
        // recompute derivative at the final node
        double pm1 = 1.0, p = x;
        for (int j = 2; j <= n; ++j) {
            double pj = ((2 * j - 1) * x * p - (j - 1) * pm1) / j;
            pm1 = p;
            p = pj;
        }
        if (n == 1) { p = x; pm1 = 1.0; }
        dpn = n * (pm1 - x * p) / (1.0 - x * x);
        t[i] = 0.5 * (x + 1.0);
        w[i] = 1.0 / ((1.0 - x * x) * dpn * dpn);
    }
}

// Jacobi polynomial P_n^{(a,0)}(x) and its derivative.
static void jacobi_a0(int n, double a, double x, double* p, double* dp) {
    // P_n^{(a,b)} by the standard three-term recurrence (b = 0 here), and
    // d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)} evaluated the same way.
    auto eval = [](int n_, double a_, double b_, double x_) {
        if (n_ == 0) return 1.0;
        double p0 = 1.0;
        double p1 = 0.5 * (a_ - b_) + 0.5 * (a_ + b_ + 2.0) * x_;
        for (int j = 1; j < n_; ++j) {
            double c = 2.0 * j + a_ + b_;
            double a1 = 2.0 * (j + 1) * (j + a_ + b_ + 1) * c;
            double a2 = (c + 1) * (a_ * a_ - b_ * b_);
            double a3 = c * (c + 1) * (c + 2);
            double a4 = 2.0 * (j + a_) * (j + b_) * (c + 2);
            double p2 = ((a2 + a3 * x_) * p1 - a4 * p0) / a1;
            p0 = p1;
            p1 = p2;
        }
        return p1;
    };
    *p = eval(n, a, 0.0, x);
    *dp = n == 0 ? 0.0 : 0.5 * (n + a + 1.0) * eval(n - 1, a + 1.0, 1.0, x);
}

// Orthonormal Dubiner basis on the reference triangle T = {r,s >= 0, r+s <= 1}
// (int_T phi_i phi_j = delta_ij), ordered by total degree d = p+q, then p:
//   phi_pq = sqrt(2(2p+1)(p+q+1)) P_p(a) (1-s)^p P_q^{(2p+1,0)}(2s-1),
//   a = 2r/(1-s) - 1  (collapsed coordinate).
// Gradients by the chain rule; points must have s < 1 (all rules here do).
void dg_dubiner(int k, double r, double s, double* phi, double* dr, double* ds) {
    double oms = 1.0 - s;
    double a = 2.0 * r / oms - 1.0;
    double b = 2.0 * s - 1.0;
    int m = 0;
    for (int d = 0; d <= k; ++d)
        for (int p = 0; p <= d; ++p) {
            int q = d - p;
            double A, dA, B, dB;
            jacobi_a0(p, 0.0, a, &A, &dA);
            jacobi_a0(q, 2.0 * p + 1.0, b, &B, &dB);
            double norm = sqrt(2.0 * (2 * p + 1) * (p + q + 1));
            double omsp = pow(oms, p);
            double omsp1 = p > 0 ? pow(oms, p - 1) : 0.0;
            phi[m] = norm * A * omsp * B;
            if (dr) dr[m] = p > 0 ? norm * 2.0 * dA * omsp1 * B : 0.0;
            if (ds) {
                // d/ds: da/ds = (a+1)/(1-s), d(1-s)^p/ds = -p(1-s)^(p-1), db/ds = 2
                double t1 = p > 0 ? (dA * (a + 1.0) - p * A) * omsp1 * B : 0.0;
                ds[m] = norm * (t1 + 2.0 * A * omsp * dB);
            }
            ++m;
        }
}

TabLayout dg_table_layout(int k) {
    TabLayout L{};
    L.k = k;
    L.nb = dg_nb(k);
    L.nq = k + 2;
    L.qk = L.nq * L.nq;
    L.qerr = (k + 4) * (k + 4);
    int o = 0;
    L.vol_w = o; o += L.qk;
    L.vol_r = o; o += L.qk;
    L.vol_s = o; o += L.qk;
    L.vol_phi = o; o += L.qk * L.nb;
    L.vol_dr = o; o += L.qk * L.nb;
    L.vol_ds = o; o += L.qk * L.nb;
    L.face_w = o; o += L.nq;
    L.face_r = o; o += 3 * L.nq;
    L.face_s = o; o += 3 * L.nq;
    L.face_phi = o; o += 3 * L.nq * L.nb;
    L.face_dr = o; o += 3 * L.nq * L.nb;
    L.face_ds = o; o += 3 * L.nq * L.nb;
    L.err_w = o; o += L.qerr;
    L.err_r = o; o += L.qerr;
    L.err_s = o; o += L.qerr;
    L.err_phi = o; o += L.qerr * L.nb;
    L.ct = o; o += DG_NCT * L.nb * L.nb;
    L.total = o;
    return L;
}

// Reference contraction matrices of the element-row assembly.  With affine
// elements every integrand of Eq. (ds) is a reference-element integral times
// per-element factors: for grad phi = J^-T grad^ phi^ the diffusion term
// needs S_ab[i][j] = sum_q w_q d_a phi_j d_b phi_i (a, b in {r, s}); the
// convection term with b affine in x, hence in (r, s), needs C_am[i][j] =
// sum_q w_q mu_m d_a phi_j phi_i with mu in {1, r, s}; the reaction term the
// mass matrix M.  On face f (Gauss points q, weights w_q of [0,1]):
// E_fa[i][j] = sum_q w_q d_a phi_j phi_i and M_f, and for the neighbour's
// basis seen at the same points (its face nf, points in reverse order, psi):
// X_a = sum w d_a psi_j phi_i, Y_a = sum w d_a phi_i psi_j, Z = sum w psi_j phi_i.
static void dg_build_contractions(const TabLayout& L, double* T) {
    const int nb = L.nb, nq = L.nq, nb2 = nb * nb;
    double* C = T + L.ct;
    auto vphi = [&](int q, int i) { return T[L.vol_phi + q * nb + i]; };
    auto vd = [&](int a, int q, int i) { return T[(a == 0 ? L.vol_dr : L.vol_ds) + q * nb + i]; };
    auto fphi = [&](int f, int q, int i) { return T[L.face_phi + (f * nq + q) * nb + i]; };
    auto fd = [&](int a, int f, int q, int i) { return T[(a == 0 ? L.face_dr : L.face_ds) + (f * nq + q) * nb + i]; };
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
            const int m = i * nb + j;
            double v[DG_NCT_VOL] = {0};
            for (int q = 0; q < L.qk; ++q) {
                const double w = T[L.vol_w + q], r = T[L.vol_r + q], s = T[L.vol_s + q];
                v[0] += w * vd(0, q, j) * vd(0, q, i);
                v[1] += w * (vd(0, q, j) * vd(1, q, i) + vd(1, q, j) * vd(0, q, i));
                v[2] += w * vd(1, q, j) * vd(1, q, i);
                const double mu[3] = {1.0, r, s};
                for (int a = 0; a < 2; ++a)
                    for (int t = 0; t < 3; ++t) v[3 + 3 * a + t] += w * mu[t] * vd(a, q, j) * vphi(q, i);
                v[9] += w * vphi(q, j) * vphi(q, i);
            }
            for (int t = 0; t < DG_NCT_VOL; ++t) C[t * nb2 + m] = v[t];
            for (int f = 0; f < 3; ++f) {
                double e[DG_NCT_SELF] = {0};
                for (int q = 0; q < nq; ++q) {
                    const double w = T[L.face_w + q];
                    e[0] += w * fd(0, f, q, j) * fphi(f, q, i);
                    e[1] += w * fd(1, f, q, j) * fphi(f, q, i);
                    e[2] += w * fphi(f, q, j) * fphi(f, q, i);
                }
                for (int t = 0; t < DG_NCT_SELF; ++t) C[(DG_NCT_VOL + DG_NCT_SELF * f + t) * nb2 + m] = e[t];
                for (int nf = 0; nf < 3; ++nf) {
                    double x[DG_NCT_CROSS] = {0};
                    for (int q = 0; q < nq; ++q) {
                        const double w = T[L.face_w + q];
                        const int qq = nq - 1 - q;
                        x[0] += w * fd(0, nf, qq, j) * fphi(f, q, i);
                        x[1] += w * fd(1, nf, qq, j) * fphi(f, q, i);
                        x[2] += w * fd(0, f, q, i) * fphi(nf, qq, j);
                        x[3] += w * fd(1, f, q, i) * fphi(nf, qq, j);
                        x[4] += w * fphi(nf, qq, j) * fphi(f, q, i);
                    }
                    const int base = DG_NCT_VOL + 3 * DG_NCT_SELF + DG_NCT_CROSS * (3 * f + nf);
                    for (int t = 0; t < DG_NCT_CROSS; ++t) C[(base + t) * nb2 + m] = x[t];
                }
            }
        }
}

// Duffy-collapsed rule: r = u (1 - v), s = v, weight wu wv (1 - v).
static void duffy(int n, double* r, double* s, double* w) {
    double t[16], tw[16];
    dg_gauss_legendre01(n, t, tw);
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            int q = b * n + a;
            r[q] = t[a] * (1.0 - t[b]);
            s[q] = t[b];
            w[q] = tw[a] * tw[b] * (1.0 - t[b]);
        }
}

void dg_build_tables(int k, double* T) {
    TabLayout L = dg_table_layout(k);
    memset(T, 0, sizeof(double) * L.total);
    duffy(L.nq, T + L.vol_r, T + L.vol_s, T + L.vol_w);
    for (int q = 0; q < L.qk; ++q)
        dg_dubiner(k, T[L.vol_r + q], T[L.vol_s + q], T + L.vol_phi + q * L.nb, T + L.vol_dr + q * L.nb,
                   T + L.vol_ds + q * L.nb);
    double t[16], tw[16];
    dg_gauss_legendre01(L.nq, t, tw);
    const double V[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    for (int q = 0; q < L.nq; ++q) T[L.face_w + q] = tw[q];
    for (int f = 0; f < 3; ++f)
        for (int q = 0; q < L.nq; ++q) {
            const double* A = V[f];
            const double* B = V[(f + 1) % 3];
            double r = A[0] + t[q] * (B[0] - A[0]);
            double s = A[1] + t[q] * (B[1] - A[1]);
            T[L.face_r + f * L.nq + q] = r;
            T[L.face_s + f * L.nq + q] = s;
            int o = (f * L.nq + q) * L.nb;
            dg_dubiner(k, r, s, T + L.face_phi + o, T + L.face_dr + o, T + L.face_ds + o);
        }
    duffy(k + 4, T + L.err_r, T + L.err_s, T + L.err_w);
    for (int q = 0; q < L.qerr; ++q)
        dg_dubiner(k, T[L.err_r + q], T[L.err_s + q], T + L.err_phi + q * L.nb, nullptr, nullptr);
    dg_build_contractions(L, T);
}

dg_status dg_ensure_tables(dg_handle* h, int k) {
    DG_WS_SCOPE(h, DG_WS_MESH);
    if (h->tab_k == k && h->tab) return DG_OK;
    TabLayout L = dg_table_layout(k);
    std::vector<double> host(L.total);
    dg_build_tables(k, host.data());
    dg_status s = dg_realloc(h, (void**)&h->tab, sizeof(double) * L.total);
    if (s != DG_OK) return s;
    DG_CK(h, cudaMemcpyAsync(h->tab, host.data(), sizeof(double) * L.total, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    h->tl = L;
    h->tab_k = k;
    return DG_OK;
}

extern "C" dg_status dg_reference_basis(int degree, int np, const double* rs, double* phi, double* dr,
                                        double* ds) {
    if (degree < 1 || degree > DG_MAXK || np < 0 || (np > 0 && (!rs || !phi))) return DG_ERR_INVALID_ARG;
    int nb = dg_nb(degree);
    for (int p = 0; p < np; ++p) {
        if (!(rs[2 * p + 1] < 1.0)) return DG_ERR_INVALID_ARG;
        dg_dubiner(degree, rs[2 * p], rs[2 * p + 1], phi + (size_t)p * nb, dr ? dr + (size_t)p * nb : nullptr,
                   ds ? ds + (size_t)p * nb : nullptr);
    }
    return DG_OK;
}

extern "C" dg_status dg_reference_rule(int which, int degree, double* rs, double* w, int* n) {
    if (degree < 1 || degree > DG_MAXK || !n) return DG_ERR_INVALID_ARG;
    TabLayout L = dg_table_layout(degree);
    std::vector<double> T(L.total);
    dg_build_tables(degree, T.data());
    int cnt, ro, so, wo;
    if (which == DG_POINTS_VOLUME) { cnt = L.qk; ro = L.vol_r; so = L.vol_s; wo = L.vol_w; }
    else if (which == DG_POINTS_BOUNDARY) { cnt = L.nq; ro = -1; so = -1; wo = L.face_w; }
    else if (which == DG_POINTS_ERROR) { cnt = L.qerr; ro = L.err_r; so = L.err_s; wo = L.err_w; }
    else return DG_ERR_INVALID_ARG;
    *n = cnt;
    double t[16], tw[16];
    if (which == DG_POINTS_BOUNDARY) dg_gauss_legendre01(L.nq, t, tw);
    for (int q = 0; q < cnt; ++q) {
        if (rs) {
            rs[2 * q] = which == DG_POINTS_BOUNDARY ? t[q] : T[ro + q];
            rs[2 * q + 1] = which == DG_POINTS_BOUNDARY ? 0.0 : T[so + q];
        }
        if (w) w[q] = T[wo + q];
    }
    return DG_OK;
}
