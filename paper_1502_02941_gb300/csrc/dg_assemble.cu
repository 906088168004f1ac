// dg_assemble.cu -- element-row ("owner computes") assembly of Stiff = D+C+R
// and of F (Eq. (ds), (dgscheme), (system) of Uzunca & Karasozen).
//
// Mapping: one CTA per tile of 32 elements.  With affine elements each block
// entry is a short sum of per-element factors times reference-element
// contraction matrices (built once per degree, staged in shared memory), plus
// the upwind terms, which are evaluated pointwise at the face points because
// min(b.n, 0) is not polynomial.  Lanes of a warp are the 32 elements of the
// tile, so every table read is a shared-memory broadcast; each block entry is
// written exactly once (no atomics, no races).
//
// Per element K, test function phi_i on K, trial phi_j (on K or on the
// neighbour L across face f), outward normal n of K, face weight w|e|:
//   volume:   eps grad phi_j.grad phi_i + (b.grad phi_j) phi_i + alpha phi_j phi_i
//   interior: (K,K) += -1/2 eps (grad phi_j.n) phi_i + kappa/2 eps (grad phi_i.n) phi_j
//                       + sigma eps/h_e phi_j phi_i - min(b.n,0) phi_j phi_i
//             (K,L) += -1/2 eps (grad psi_j.n) phi_i - kappa/2 eps (grad phi_i.n) psi_j
//                       - sigma eps/h_e psi_j phi_i + min(b.n,0) psi_j phi_i
//   Dirichlet:(K,K) += -eps (grad phi_j.n) phi_i + kappa eps (grad phi_i.n) phi_j
//                       + sigma_b eps/h_e phi_j phi_i - min(b.n,0) phi_j phi_i
//   Neumann:  (K,K) += -min(b.n,0) phi_j phi_i
// which is the jump/average form of Eq. (ds) with [v] = v_K n_K + v_L n_L and
// {q} = (q_K + q_L)/2 restricted to test functions supported on K; the upwind
// weight min(b.n,0) selects dK^- pointwise at each quadrature point.
#include "dg_internal.cuh"

struct AsmArgs {
    const double* geo;
    const int* nbr;
    const int* nface;
    const int* ftype;
    const int* bidx;
    const double* tab;
    TabLayout L;
    int ne;
    double eps, alpha, kappa, sig_int, sig_bdry;
    double b0;        // superpenalisation: the penalty terms carry sigma eps / |e|^b0
    double b[6];
    double* A64;
    float* A32;
    __nv_bfloat16* A16;
    // per-instance coefficients of a batch (NULL for one instance): element K
    // uses icoef[DG_ICOEF * inst[K] + ...] = eps, alpha, b[6], sigma_int, sigma_bdry
    const int* inst;
    const double* icoef;
    // RHS data
    const double* f;
    double f_const;
    const double* gD;
    double gD_const;
    const double* gN;
    double gN_const;
    double* F;
};

__device__ __forceinline__ double gload(const double* geo, int field, int ne, int K) {
    return __ldg(geo + (size_t)field * ne + K);
}

// Stage the volume and face tables of degree K_DEG into shared memory.
template <int K_DEG>
__device__ __forceinline__ void stage_tables(const double* __restrict__ tab, const TabLayout& L, double* sm) {
    // copy [vol_w, face_ds end) contiguous region
    int n = L.err_w;  // everything before the error-rule tables
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[t] = tab[t];
    __syncthreads();
}

// Per-element factors of the reference contractions (see dg_tables.cu):
// 10 volume factors, then per face f: sA_r, sA_s (trial gradient . n on the
// test function), sB_r, sB_s (test gradient . n on the trial function), sC
// (penalty), xA_r, xA_s, xB_r, xB_s, xC (the same for the neighbour block),
// xU (1 on interior faces), u_q = -w_q |e| min(b.n, 0) at the face points.
template <int NQ>
struct CoefIdx {
    static constexpr int FACE = 11 + NQ;
    static constexpr int N = 10 + 3 * FACE;
};

// Factors of the reference contractions, one thread per (element, part):
// part 0 the volume factors, parts 1..3 the factors of face part-1.  Written
// to the SoA array fac [CoefIdx::N][ne] (and the neighbour's face to nfo [3][ne]).
template <int K_DEG>
__global__ void __launch_bounds__(256) k_asm_factors(const AsmArgs a, double* __restrict__ fac, int* __restrict__ nfo) {
    constexpr int NQ = K_DEG + 2;
    using CI = CoefIdx<NQ>;
    const int ne = a.ne;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4L * ne) return;
    const int part = (int)(t / ne), K = (int)(t - (long)part * ne);
    const TabLayout& L = a.L;
    const double* fw = a.tab + L.face_w;
    const double* fr = a.tab + L.face_r;
    const double* fs = a.tab + L.face_s;
    const size_t sne = (size_t)ne;
    double* c = fac + K;               // c[idx * ne]
    {
        {
            const double x0 = gload(a.geo, G_X0, ne, K), y0 = gload(a.geo, G_Y0, ne, K);
            const double j00 = gload(a.geo, G_J00, ne, K), j01 = gload(a.geo, G_J01, ne, K);
            const double j10 = gload(a.geo, G_J10, ne, K), j11 = gload(a.geo, G_J11, ne, K);
            const double i00 = gload(a.geo, G_I00, ne, K), i01 = gload(a.geo, G_I01, ne, K);
            const double i10 = gload(a.geo, G_I10, ne, K), i11 = gload(a.geo, G_I11, ne, K);
            const double det = gload(a.geo, G_DET, ne, K);
            double eps = a.eps, alpha = a.alpha, sig_int = a.sig_int, sig_bdry = a.sig_bdry;
            double bc[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) bc[t] = a.b[t];
            if (a.inst) {
                const double* ci = a.icoef + (size_t)DG_ICOEF * a.inst[K];
                eps = ci[0];
                alpha = ci[1];
#pragma unroll
                for (int t = 0; t < 6; ++t) bc[t] = ci[2 + t];
                sig_int = ci[8];
                sig_bdry = ci[9];
            }
            if (part == 0) {
                // diffusion: grad phi_j . grad phi_i = sum_ab G_ab d_a phi_j d_b phi_i, G = Jinv Jinv^T
                c[0 * sne] = eps * det * (i00 * i00 + i01 * i01);
                c[1 * sne] = eps * det * (i00 * i10 + i01 * i11);
                c[2 * sne] = eps * det * (i10 * i10 + i11 * i11);
                // convection: b(x(r,s)) affine in (r, s); beta_a = sum_c Jinv[a][c] b_c
                const double bx0 = bc[0] + bc[1] * x0 + bc[2] * y0, bxr = bc[1] * j00 + bc[2] * j10,
                             bxs = bc[1] * j01 + bc[2] * j11;
                const double by0 = bc[3] + bc[4] * x0 + bc[5] * y0, byr = bc[4] * j00 + bc[5] * j10,
                             bys = bc[4] * j01 + bc[5] * j11;
                c[3 * sne] = det * (i00 * bx0 + i01 * by0);
                c[4 * sne] = det * (i00 * bxr + i01 * byr);
                c[5 * sne] = det * (i00 * bxs + i01 * bys);
                c[6 * sne] = det * (i10 * bx0 + i11 * by0);
                c[7 * sne] = det * (i10 * bxr + i11 * byr);
                c[8 * sne] = det * (i10 * bxs + i11 * bys);
                c[9 * sne] = alpha * det;
            } else {
                const int f = part - 1;
                const double dV[3][2] = {{1.0, 0.0}, {-1.0, 1.0}, {0.0, -1.0}};
                const int type = __ldg(a.ftype + (size_t)f * ne + K);
                const int Ln = __ldg(a.nbr + (size_t)f * ne + K);
                const int nf = type == 0 ? __ldg(a.nface + (size_t)f * ne + K) : 0;
                const double tx = j00 * dV[f][0] + j01 * dV[f][1];
                const double ty = j10 * dV[f][0] + j11 * dV[f][1];
                const double len = sqrt(tx * tx + ty * ty);
                const double nx = ty / len, ny = -tx / len;
                // penalty sigma eps / h_e^b0 with h_e = |e|, integrated over |e|
                const double pfac = a.b0 == 1.0 ? 1.0 : pow(len, 1.0 - a.b0);
                const double nu_r = i00 * nx + i01 * ny, nu_s = i10 * nx + i11 * ny;
                const double fac1 = type == 0 ? -0.5 : (type == 1 ? -1.0 : 0.0);
                const double fac2 = type == 0 ? 0.5 : (type == 1 ? 1.0 : 0.0);
                const double sig = type == 0 ? sig_int : (type == 1 ? sig_bdry : 0.0);
                double* cf = c + (10 + f * CI::FACE) * sne;
                cf[0 * sne] = fac1 * eps * len * nu_r;
                cf[1 * sne] = fac1 * eps * len * nu_s;
                cf[2 * sne] = fac2 * a.kappa * eps * len * nu_r;
                cf[3 * sne] = fac2 * a.kappa * eps * len * nu_s;
                cf[4 * sne] = sig * eps * pfac;
                double lnr = 0.0, lns = 0.0;
                if (type == 0) {
                    const double li00 = gload(a.geo, G_I00, ne, Ln), li01 = gload(a.geo, G_I01, ne, Ln);
                    const double li10 = gload(a.geo, G_I10, ne, Ln), li11 = gload(a.geo, G_I11, ne, Ln);
                    lnr = li00 * nx + li01 * ny;
                    lns = li10 * nx + li11 * ny;
                }
                const double in = type == 0 ? 1.0 : 0.0;
                cf[5 * sne] = -0.5 * in * eps * len * lnr;
                cf[6 * sne] = -0.5 * in * eps * len * lns;
                cf[7 * sne] = -0.5 * in * a.kappa * eps * len * nu_r;
                cf[8 * sne] = -0.5 * in * a.kappa * eps * len * nu_s;
                cf[9 * sne] = -in * sig_int * eps * pfac;
                cf[10 * sne] = in;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const double x = x0 + j00 * fr[f * NQ + q] + j01 * fs[f * NQ + q];
                    const double y = y0 + j10 * fr[f * NQ + q] + j11 * fs[f * NQ + q];
                    const double bn = (bc[0] + bc[1] * x + bc[2] * y) * nx + (bc[3] + bc[4] * x + bc[5] * y) * ny;
                    const double up = bn < 0.0 ? bn : 0.0;
                    cf[(11 + q) * sne] = -fw[q] * len * up;
                }
                nfo[(size_t)f * ne + K] = nf;
            }
        }
    }
}

// Element-row assembly: one CTA per tile of 32 elements; the tile's factors
// are staged in shared memory, then warp w computes block entries m = w, w + 8,
// ... of the four blocks of its 32 elements (lane = element) as sums of factor
// x reference matrix (shared-memory broadcasts) plus the pointwise upwind sums,
// and writes them into the tile-interleaved block-ELL copies.  Each entry is
// written once.
template <int K_DEG>
__global__ void __launch_bounds__(256) k_assemble(const AsmArgs a, const double* __restrict__ fac,
                                                  const int* __restrict__ nfo) {
    constexpr int NB = dg_nb(K_DEG);
    constexpr int NQ = K_DEG + 2;
    constexpr int NB2 = NB * NB;
    using CI = CoefIdx<NQ>;
    constexpr int NCT = DG_NCT * NB2;
    constexpr int NFB = NQ + 6 * NQ + 3 * NQ * NB;   // face_w, face_r, face_s, face_phi
    extern __shared__ double sm[];
    double* sct = sm;                  // contraction matrices
    double* sfb = sct + NCT;           // face rule + basis at face points
    double* scf = sfb + NFB;           // factors [CI::N][32]
    int* snf = reinterpret_cast<int*>(scf + CI::N * 32);   // neighbour's face [3][32]
    const TabLayout& L = a.L;
    for (int t = threadIdx.x; t < NCT; t += blockDim.x) sct[t] = a.tab[L.ct + t];
    for (int t = threadIdx.x; t < NFB; t += blockDim.x) sfb[t] = a.tab[L.face_w + t];
    const int ne = a.ne;
    const int tile = blockIdx.x;
    for (int t = threadIdx.x; t < CI::N * 32; t += blockDim.x) {
        const int idx = t >> 5, K = tile * 32 + (t & 31);
        scf[t] = K < ne ? fac[(size_t)idx * ne + K] : 0.0;
    }
    if (threadIdx.x < 96) {
        const int f = threadIdx.x >> 5, K = tile * 32 + (threadIdx.x & 31);
        snf[threadIdx.x] = K < ne ? nfo[(size_t)f * ne + K] : 0;
    }
    const double* fp = sfb + 7 * NQ;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = tile * 32 + lane;
    const double* c = scf + lane;
    for (int m = warp; m < NB2; m += 8) {
        const int i = m / NB, j = m - (m / NB) * NB;
        const int mt = j * NB + i;
        double out[4];
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < DG_NCT_VOL; ++t) acc = fma(c[t * 32], sct[t * NB2 + m], acc);
        out[1] = out[2] = out[3] = 0.0;
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            const double* cf = c + (10 + f * CI::FACE) * 32;
            const double* E = sct + (DG_NCT_VOL + DG_NCT_SELF * f) * NB2;
            acc = fma(cf[0 * 32], E[m], acc);
            acc = fma(cf[1 * 32], E[NB2 + m], acc);
            acc = fma(cf[2 * 32], E[mt], acc);
            acc = fma(cf[3 * 32], E[NB2 + mt], acc);
            acc = fma(cf[4 * 32], E[2 * NB2 + m], acc);
            const int nf = snf[f * 32 + lane];
            const double* X = sct + (DG_NCT_VOL + 3 * DG_NCT_SELF + DG_NCT_CROSS * (3 * f + nf)) * NB2;
            double cr = cf[5 * 32] * X[m];
            cr = fma(cf[6 * 32], X[NB2 + m], cr);
            cr = fma(cf[7 * 32], X[2 * NB2 + m], cr);
            cr = fma(cf[8 * 32], X[3 * NB2 + m], cr);
            cr = fma(cf[9 * 32], X[4 * NB2 + m], cr);
            double us = 0.0, ux = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double uq = cf[(11 + q) * 32];
                const double pi = fp[(f * NQ + q) * NB + i];
                us = fma(uq * pi, fp[(f * NQ + q) * NB + j], us);
                ux = fma(uq * pi, fp[(nf * NQ + NQ - 1 - q) * NB + j], ux);
            }
            acc += us;
            const double xo = fma(-cf[10 * 32], ux, cr);
            if (f == 0) out[1] = xo;
            else if (f == 1) out[2] = xo;
            else out[3] = xo;
        }
        out[0] = acc;
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
            if (a.A64) a.A64[dg_blk_index<double>(K, s2, m, NB, 4)] = out[s2];
            if (a.A32) a.A32[dg_blk_index<float>(K, s2, m, NB, 4)] = (float)out[s2];
            if (a.A16) a.A16[dg_blk_index<__nv_bfloat16>(K, s2, m, NB, 4)] = __double2bfloat16(out[s2]);
        }
    }
    // chunk padding after nb^2: warp s clears slot s
    if (warp < 4) {
        const int s2 = warp;
        if (a.A64) for (int mm = NB2; mm < dg_chunks<double>(NB) * 2; ++mm) a.A64[dg_blk_index<double>(K, s2, mm, NB, 4)] = 0.0;
        if (a.A32) for (int mm = NB2; mm < dg_chunks<float>(NB) * 4; ++mm) a.A32[dg_blk_index<float>(K, s2, mm, NB, 4)] = 0.0f;
        if (a.A16) for (int mm = NB2; mm < dg_chunks<__nv_bfloat16>(NB) * 8; ++mm)
            a.A16[dg_blk_index<__nv_bfloat16>(K, s2, mm, NB, 4)] = __double2bfloat16(0.0);
    }
}

template <int K_DEG>
static size_t assemble_smem() {  // shared memory of k_assemble
    constexpr int NB = dg_nb(K_DEG), NQ = K_DEG + 2;
    return sizeof(double) * (DG_NCT * NB * NB + 7 * NQ + 3 * NQ * NB + CoefIdx<NQ>::N * 32) + sizeof(int) * 96;
}

// F_K[i]: one warp per (tile, i), lanes = elements.
template <int K_DEG>
__global__ void __launch_bounds__(256) k_rhs(const AsmArgs a) {
    constexpr int NB = dg_nb(K_DEG);
    constexpr int NQ = K_DEG + 2;
    constexpr int QK = NQ * NQ;
    extern __shared__ double sm[];
    const TabLayout& L = a.L;
    stage_tables<K_DEG>(a.tab, L, sm);
    const int lane = threadIdx.x & 31;
    const long gw = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ntiles = (a.ne + 31) >> 5;
    if (gw >= (long)ntiles * NB) return;
    const int tile = (int)(gw / NB);
    const int i = (int)(gw - (long)tile * NB);
    const int K = tile * 32 + lane;
    const int ne = a.ne;
    if (K >= ne) return;
    const double x0 = gload(a.geo, G_X0, ne, K), y0 = gload(a.geo, G_Y0, ne, K);
    const double j00 = gload(a.geo, G_J00, ne, K), j01 = gload(a.geo, G_J01, ne, K);
    const double j10 = gload(a.geo, G_J10, ne, K), j11 = gload(a.geo, G_J11, ne, K);
    const double i00 = gload(a.geo, G_I00, ne, K), i01 = gload(a.geo, G_I01, ne, K);
    const double i10 = gload(a.geo, G_I10, ne, K), i11 = gload(a.geo, G_I11, ne, K);
    const double det = gload(a.geo, G_DET, ne, K);
    double eps = a.eps, sig_bdry = a.sig_bdry;
    double bc[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) bc[t] = a.b[t];
    if (a.inst) {
        const double* c = a.icoef + (size_t)DG_ICOEF * a.inst[K];
        eps = c[0];
#pragma unroll
        for (int t = 0; t < 6; ++t) bc[t] = c[2 + t];
        sig_bdry = c[9];
    }
    double acc = 0.0;
    for (int q = 0; q < QK; ++q) {
        const double fv = a.f ? __ldg(a.f + (size_t)K * QK + q) : a.f_const;
        acc += sm[L.vol_w + q] * det * fv * sm[L.vol_phi + q * NB + i];
    }
    const double dV[3][2] = {{1.0, 0.0}, {-1.0, 1.0}, {0.0, -1.0}};
    for (int f = 0; f < 3; ++f) {
        const int type = __ldg(a.ftype + (size_t)f * ne + K);
        if (type == 0) continue;
        const int b = __ldg(a.bidx + (size_t)f * ne + K);
        const double tx = j00 * dV[f][0] + j01 * dV[f][1];
        const double ty = j10 * dV[f][0] + j11 * dV[f][1];
        const double len = sqrt(tx * tx + ty * ty);
        const double nx = ty / len, ny = -tx / len;
        const double he = a.b0 == 1.0 ? len : pow(len, a.b0);   // h_e^b0, h_e = |e|
        for (int q = 0; q < NQ; ++q) {
            const double w = sm[L.face_w + q] * len;
            const int o = (f * NQ + q) * NB + i;
            const double pi = sm[L.face_phi + o];
            const double gin = (i00 * sm[L.face_dr + o] + i10 * sm[L.face_ds + o]) * nx +
                               (i01 * sm[L.face_dr + o] + i11 * sm[L.face_ds + o]) * ny;
            const double x = x0 + j00 * sm[L.face_r + f * NQ + q] + j01 * sm[L.face_s + f * NQ + q];
            const double y = y0 + j10 * sm[L.face_r + f * NQ + q] + j11 * sm[L.face_s + f * NQ + q];
            const double bn = (bc[0] + bc[1] * x + bc[2] * y) * nx + (bc[3] + bc[4] * x + bc[5] * y) * ny;
            const double up = bn < 0.0 ? bn : 0.0;
            const double gD = a.gD ? __ldg(a.gD + (size_t)b * NQ + q) : a.gD_const;
            if (type == 1) acc += w * gD * (sig_bdry * eps / he * pi + a.kappa * eps * gin);
            acc -= w * up * gD * pi;
            if (type == 2) {
                const double gN = a.gN ? __ldg(a.gN + (size_t)b * NQ + q) : a.gN_const;
                acc += w * gN * pi;
            }
        }
    }
    a.F[(size_t)K * NB + i] = acc;
}

// ---------------------------------------------------------------------------
// variable diffusion eps(x, y) (the paper's fdiff, evaluated at the points)
// ---------------------------------------------------------------------------
// Every term of Eq. (ds) that holds eps is linear in it, so with a pointwise
// eps the operator is the eps = 0 assembly plus the terms below, which this
// kernel adds into the f64 blocks and F by quadrature with eps at each point:
//   volume  (K,K)   += int eps grad phi_j . grad phi_i
//   interior(K,K)   += int eps [-1/2 (grad phi_j.n) phi_i + kappa/2 (grad phi_i.n) phi_j
//                               + sigma/h_e^b0 phi_j phi_i]
//           (K,L)   += int eps [-1/2 (grad psi_j.n) phi_i - kappa/2 (grad phi_i.n) psi_j
//                               - sigma/h_e^b0 psi_j phi_i]
//   Dirichlet (K,K) += int eps [-(grad phi_j.n) phi_i + kappa (grad phi_i.n) phi_j
//                               + sigma_b/h_e^b0 phi_j phi_i]
//   Dirichlet F_i   += int gD eps (sigma_b/h_e^b0 phi_i + kappa grad phi_i.n)
// (the jump/average form of the constant-eps kernels above, A-1 sign).  One
// CTA per 32-element tile: lanes are elements, warps run over the entries
// (i, j) of the four blocks and then over F_i.  On an interior edge eps at a
// point is the mean of the two elements' values there.
template <int K_DEG>
__global__ void __launch_bounds__(256) k_diff_var(const AsmArgs a, const double* __restrict__ eps_q,
                                                  const double* __restrict__ eps_f) {
    constexpr int NB = dg_nb(K_DEG);
    constexpr int NQ = K_DEG + 2;
    constexpr int QK = NQ * NQ;
    constexpr int NB2 = NB * NB;
    extern __shared__ double sm[];
    const TabLayout& L = a.L;
    double* se = sm + L.err_w;          // eps at the tile's volume points [QK][32]
    double* sf = se + QK * 32;          // eps on the tile's faces [3][NQ][32]
    for (int t = threadIdx.x; t < L.err_w; t += blockDim.x) sm[t] = a.tab[t];
    const int ne = a.ne;
    const int tile = blockIdx.x;
    for (int t = threadIdx.x; t < QK * 32; t += blockDim.x) {
        const int q = t >> 5, K = tile * 32 + (t & 31);
        se[t] = K < ne ? eps_q[(size_t)K * QK + q] : 0.0;
    }
    for (int t = threadIdx.x; t < 3 * NQ * 32; t += blockDim.x) {
        const int fq = t >> 5, K = tile * 32 + (t & 31);
        const int f = fq / NQ, q = fq - f * NQ;
        double v = 0.0;
        if (K < ne) {
            v = eps_f[((size_t)K * 3 + f) * NQ + q];
            if (__ldg(a.ftype + (size_t)f * ne + K) == 0) {
                const int Ln = __ldg(a.nbr + (size_t)f * ne + K), nf = __ldg(a.nface + (size_t)f * ne + K);
                v = 0.5 * (v + eps_f[((size_t)Ln * 3 + nf) * NQ + (NQ - 1 - q)]);
            }
        }
        sf[t] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = tile * 32 + lane;
    if (K >= ne) return;
    const double j00 = gload(a.geo, G_J00, ne, K), j01 = gload(a.geo, G_J01, ne, K);
    const double j10 = gload(a.geo, G_J10, ne, K), j11 = gload(a.geo, G_J11, ne, K);
    const double i00 = gload(a.geo, G_I00, ne, K), i01 = gload(a.geo, G_I01, ne, K);
    const double i10 = gload(a.geo, G_I10, ne, K), i11 = gload(a.geo, G_I11, ne, K);
    const double det = gload(a.geo, G_DET, ne, K);
    const double grr = i00 * i00 + i01 * i01, grs = i00 * i10 + i01 * i11, gss = i10 * i10 + i11 * i11;
    const double* vw = sm + L.vol_w;
    const double* vdr = sm + L.vol_dr;
    const double* vds = sm + L.vol_ds;
    const double* fw = sm + L.face_w;
    const double* fphi = sm + L.face_phi;
    const double* fdr = sm + L.face_dr;
    const double* fds = sm + L.face_ds;
    const double dV[3][2] = {{1.0, 0.0}, {-1.0, 1.0}, {0.0, -1.0}};
    for (int m = warp; m < NB2 + NB; m += 8) {
        const bool rhs = m >= NB2;
        const int i = rhs ? m - NB2 : m / NB, j = rhs ? 0 : m - (m / NB) * NB;
        double out[4] = {0.0, 0.0, 0.0, 0.0};
        if (!rhs) {
            for (int q = 0; q < QK; ++q) {
                const double dri = vdr[q * NB + i], dsi = vds[q * NB + i];
                const double drj = vdr[q * NB + j], dsj = vds[q * NB + j];
                const double g = grr * drj * dri + grs * (drj * dsi + dsj * dri) + gss * dsj * dsi;
                out[0] = fma(vw[q] * det * se[q * 32 + lane], g, out[0]);
            }
        }
        for (int f = 0; f < 3; ++f) {
            const int type = __ldg(a.ftype + (size_t)f * ne + K);
            if (type == 2 || (rhs && type != 1)) continue;
            const double tx = j00 * dV[f][0] + j01 * dV[f][1];
            const double ty = j10 * dV[f][0] + j11 * dV[f][1];
            const double len = sqrt(tx * tx + ty * ty);
            const double nx = ty / len, ny = -tx / len;
            const double ph = a.b0 == 1.0 ? 1.0 / len : pow(len, -a.b0);   // 1 / h_e^b0
            const double sig = type == 0 ? a.sig_int : a.sig_bdry;
            int Ln = -1, nf = 0;
            double l00 = 0.0, l01 = 0.0, l10 = 0.0, l11 = 0.0;
            if (type == 0) {
                Ln = __ldg(a.nbr + (size_t)f * ne + K);
                nf = __ldg(a.nface + (size_t)f * ne + K);
                l00 = gload(a.geo, G_I00, ne, Ln);
                l01 = gload(a.geo, G_I01, ne, Ln);
                l10 = gload(a.geo, G_I10, ne, Ln);
                l11 = gload(a.geo, G_I11, ne, Ln);
            }
            const int b = rhs ? __ldg(a.bidx + (size_t)f * ne + K) : -1;
            double kk = 0.0, kl = 0.0;
            for (int q = 0; q < NQ; ++q) {
                const double w = fw[q] * len * sf[(f * NQ + q) * 32 + lane];
                const int oi = (f * NQ + q) * NB + i;
                const double pi = fphi[oi];
                const double gi = (i00 * fdr[oi] + i10 * fds[oi]) * nx + (i01 * fdr[oi] + i11 * fds[oi]) * ny;
                if (rhs) {
                    const double gD = a.gD ? __ldg(a.gD + (size_t)b * NQ + q) : a.gD_const;
                    kk = fma(w * gD, sig * ph * pi + a.kappa * gi, kk);
                    continue;
                }
                const int oj = (f * NQ + q) * NB + j;
                const double pj = fphi[oj];
                const double gj = (i00 * fdr[oj] + i10 * fds[oj]) * nx + (i01 * fdr[oj] + i11 * fds[oj]) * ny;
                if (type == 0) {
                    kk = fma(w, -0.5 * gj * pi + 0.5 * a.kappa * gi * pj + sig * ph * pj * pi, kk);
                    const int ol = (nf * NQ + NQ - 1 - q) * NB + j;
                    const double psj = fphi[ol];
                    const double gl = (l00 * fdr[ol] + l10 * fds[ol]) * nx + (l01 * fdr[ol] + l11 * fds[ol]) * ny;
                    kl = fma(w, -0.5 * gl * pi - 0.5 * a.kappa * gi * psj - sig * ph * psj * pi, kl);
                } else {
                    kk = fma(w, -gj * pi + a.kappa * gi * pj + sig * ph * pj * pi, kk);
                }
            }
            out[0] += kk;
            if (!rhs && type == 0) out[1 + f] = kl;
        }
        if (rhs) {
            a.F[(size_t)K * NB + i] += out[0];
        } else {
            a.A64[dg_blk_index<double>(K, 0, m, NB, 4)] += out[0];
            for (int f = 0; f < 3; ++f)
                if (out[1 + f] != 0.0) a.A64[dg_blk_index<double>(K, 1 + f, m, NB, 4)] += out[1 + f];
        }
    }
}

// The f32 / bf16 block copies rounded from the f64 blocks (after k_diff_var).
template <int NB>
__global__ void __launch_bounds__(256) k_round_copies(const double* __restrict__ A64, float* A32, __nv_bfloat16* A16,
                                                      int ne) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)ne * 4 * NB * NB) return;
    const int K = (int)(t / (4 * NB * NB));
    const int r = (int)(t - (long)K * 4 * NB * NB);
    const int s = r / (NB * NB), m = r - s * NB * NB;
    const double v = A64[dg_blk_index<double>(K, s, m, NB, 4)];
    if (A32) A32[dg_blk_index<float>(K, s, m, NB, 4)] = (float)v;
    if (A16) A16[dg_blk_index<__nv_bfloat16>(K, s, m, NB, 4)] = __double2bfloat16(v);
}

dg_status dg_launch_assemble(dg_handle* h, const dg_coeffs* c, double kappa, double sig_int, double sig_bdry) {
    const int k = h->p.degree;
    const int nb = dg_nb(k);
    AsmArgs a{};
    a.geo = h->geo;
    a.nbr = h->nbr;
    a.nface = h->nface;
    a.ftype = h->ftype;
    a.bidx = h->bidx;
    a.tab = h->tab;
    a.L = h->tl;
    a.ne = h->ne;
    a.eps = c->eps;
    a.alpha = c->alpha;
    a.kappa = kappa;
    a.b0 = h->p.b0;
    a.sig_int = sig_int;
    a.sig_bdry = sig_bdry;
    for (int t = 0; t < 6; ++t) a.b[t] = c->b[t];
    a.A64 = (h->p.store & DG_STORE_F64) ? h->A64 : nullptr;
    a.A32 = (h->p.store & DG_STORE_F32) ? h->A32 : nullptr;
    a.A16 = (h->p.store & DG_STORE_BF16) ? h->A16 : nullptr;
    a.f = c->f;
    a.f_const = c->f_const;
    a.gD = c->gD;
    a.gD_const = c->gD_const;
    a.gN = c->gN;
    a.gN_const = c->gN_const;
    a.F = h->F;
    a.inst = h->b_inst_active ? h->b_inst : nullptr;
    a.icoef = h->b_inst_active ? h->b_icoef : nullptr;
    const size_t smem = sizeof(double) * h->tl.err_w;
    const long warps_r = (long)h->ntiles * nb;
    const unsigned ga = (unsigned)h->ntiles, gr = (unsigned)((warps_r + 7) / 8);
    const unsigned gf = (unsigned)((4L * h->ne + 255) / 256);
    // factor scratch: [CoefIdx::N][ne] f64 + [3][ne] int
    const int ncoef = 10 + 3 * (11 + k + 2);
    dg_status s = dg_scratch(h, sizeof(double) * (size_t)ncoef * h->ne + sizeof(int) * 3 * (size_t)h->ne + 16);
    if (s != DG_OK) return s;
    double* fac = h->scratch;
    int* nfo = reinterpret_cast<int*>(fac + (size_t)ncoef * h->ne);
    switch (k) {
        case 1:
            DG_CK(h, cudaFuncSetAttribute(k_assemble<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble_smem<1>()));
            k_asm_factors<1><<<gf, 256, 0, h->stream>>>(a, fac, nfo);
            k_assemble<1><<<ga, 256, assemble_smem<1>(), h->stream>>>(a, fac, nfo);
            k_rhs<1><<<gr, 256, smem, h->stream>>>(a);
            break;
        case 2:
            DG_CK(h, cudaFuncSetAttribute(k_assemble<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble_smem<2>()));
            k_asm_factors<2><<<gf, 256, 0, h->stream>>>(a, fac, nfo);
            k_assemble<2><<<ga, 256, assemble_smem<2>(), h->stream>>>(a, fac, nfo);
            k_rhs<2><<<gr, 256, smem, h->stream>>>(a);
            break;
        case 3:
            DG_CK(h, cudaFuncSetAttribute(k_assemble<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble_smem<3>()));
            k_asm_factors<3><<<gf, 256, 0, h->stream>>>(a, fac, nfo);
            k_assemble<3><<<ga, 256, assemble_smem<3>(), h->stream>>>(a, fac, nfo);
            k_rhs<3><<<gr, 256, smem, h->stream>>>(a);
            break;
        default:
            return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += 3;
    DG_LAUNCH_CK(h);
    if (c->eps_q) {
        // pointwise eps: the kernels above ran with eps = 0 (the caller's copy
        // of the coefficients); add the eps terms, then round the copies
        const size_t dsmem = sizeof(double) * ((size_t)h->tl.err_w + 32 * (size_t)(h->tl.qk + 3 * h->tl.nq));
        const long nent = (long)h->ne * 4 * nb * nb;
        const unsigned gc = (unsigned)((nent + 255) / 256);
        switch (k) {
            case 1:
                DG_CK(h, cudaFuncSetAttribute(k_diff_var<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
                k_diff_var<1><<<ga, 256, dsmem, h->stream>>>(a, c->eps_q, c->eps_f);
                if (a.A32 || a.A16) k_round_copies<3><<<gc, 256, 0, h->stream>>>(a.A64, a.A32, a.A16, h->ne);
                break;
            case 2:
                DG_CK(h, cudaFuncSetAttribute(k_diff_var<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
                k_diff_var<2><<<ga, 256, dsmem, h->stream>>>(a, c->eps_q, c->eps_f);
                if (a.A32 || a.A16) k_round_copies<6><<<gc, 256, 0, h->stream>>>(a.A64, a.A32, a.A16, h->ne);
                break;
            case 3:
                DG_CK(h, cudaFuncSetAttribute(k_diff_var<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
                k_diff_var<3><<<ga, 256, dsmem, h->stream>>>(a, c->eps_q, c->eps_f);
                if (a.A32 || a.A16) k_round_copies<10><<<gc, 256, 0, h->stream>>>(a.A64, a.A32, a.A16, h->ne);
                break;
        }
        h->nlaunch += (a.A32 || a.A16) ? 2 : 1;
        DG_LAUNCH_CK(h);
    }
    return DG_OK;
}

extern "C" dg_status dg_assemble(dg_handle* h, const dg_coeffs* c) {
    DG_WS_SCOPE(h, DG_WS_OPERATOR);
    if (!h || !c) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    if (!(c->eps >= 0.0) || !(c->alpha == c->alpha)) return dg_fail(h, DG_ERR_INVALID_ARG, "eps must be >= 0");
    if ((c->eps_q == nullptr) != (c->eps_f == nullptr))
        return dg_fail(h, DG_ERR_INVALID_ARG, "eps_q and eps_f are given together");
    if (c->eps_q && h->b_inst_active)
        return dg_fail(h, DG_ERR_INVALID_ARG, "a pointwise eps is not read in batch mode");
    if (c->eps_q && !(h->p.store & DG_STORE_F64))
        return dg_fail(h, DG_ERR_INVALID_ARG, "a pointwise eps needs the f64 block copy (params.store)");
    dg_coeffs cv = *c;
    if (c->eps_q) cv.eps = 0.0;   // the eps terms are added pointwise after the eps = 0 assembly
    c = &cv;
    DG_CK(h, cudaSetDevice(h->device));
    const int k = h->p.degree;
    const int nb = dg_nb(k);
    dg_status s = dg_ensure_tables(h, k);
    if (s != DG_OK) return s;
    // (re)allocate block storage for the requested copies
    const size_t per_tile_slot = 16 * 32;  // bytes per chunk row of a tile
    size_t need[3] = {0, 0, 0};
    if (h->p.store & DG_STORE_F64) need[0] = (size_t)h->ntiles * 4 * dg_chunks<double>(nb) * per_tile_slot;
    if (h->p.store & DG_STORE_F32) need[1] = (size_t)h->ntiles * 4 * dg_chunks<float>(nb) * per_tile_slot;
    if (h->p.store & DG_STORE_BF16) need[2] = (size_t)h->ntiles * 4 * dg_chunks<__nv_bfloat16>(nb) * per_tile_slot;
    void** ptrs[3] = {(void**)&h->A64, (void**)&h->A32, (void**)&h->A16};
    for (int t = 0; t < 3; ++t) {
        if (need[t] != h->A_bytes[t]) {
            if ((s = dg_realloc(h, ptrs[t], need[t])) != DG_OK) return s;
            h->A_bytes[t] = need[t];
        }
    }
    if ((s = dg_ensure(h, (void**)&h->F, &h->cap_F, sizeof(double) * (size_t)h->ne * nb)) != DG_OK) return s;
    double kappa = h->p.method == DG_NIPG ? 1.0 : (h->p.method == DG_SIPG ? -1.0 : 0.0);
    double sig = h->p.sigma_int > 0.0 ? h->p.sigma_int : (h->p.method == DG_NIPG ? 1.0 : 3.0 * k * (k + 1));
    double fac = h->p.sigma_bdry_factor > 0.0 ? h->p.sigma_bdry_factor : 2.0;
    h->assembled = false;
    h->bj_ok = false;
    h->ras_ok = false;
    if ((s = dg_launch_assemble(h, c, kappa, sig, fac * sig)) != DG_OK) return s;
    h->assembled = true;
    h->asm_k = k;
    h->asm_store = h->p.store;
    h->mlp.coef[0] = c->eps;
    h->mlp.coef[1] = c->alpha;
    for (int t = 0; t < 6; ++t) h->mlp.coef[2 + t] = c->b[t];
    return DG_OK;
}
