// dg_assemble.cu -- element-row ("owner computes") assembly of Stiff = D+C+R
// and of F (Eq. (ds), (dgscheme), (system) of Uzunca & Karasozen).
//
// Mapping: one warp per (tile of 32 elements, block entry m = i*nb + j); the
// 32 lanes are the 32 elements of the tile.  Every lane of a warp therefore
// reads the same basis-table entries (shared-memory broadcast), reads its
// element's geometry with coalesced SoA loads and writes entry m of its four
// blocks into the tile-interleaved block-ELL layout (16-byte stride between
// lanes).  Each block entry is written exactly once: no atomics, no races.
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

template <int K_DEG>
__global__ void __launch_bounds__(256) k_assemble(const AsmArgs a) {
    constexpr int NB = dg_nb(K_DEG);
    constexpr int NQ = K_DEG + 2;
    constexpr int QK = NQ * NQ;
    constexpr int NB2 = NB * NB;
    extern __shared__ double sm[];
    const TabLayout& L = a.L;
    stage_tables<K_DEG>(a.tab, L, sm);

    const int lane = threadIdx.x & 31;
    const long gw = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ntiles = (a.ne + 31) >> 5;
    if (gw >= (long)ntiles * NB2) return;
    const int tile = (int)(gw / NB2);
    const int m = (int)(gw - (long)tile * NB2);
    const int i = m / NB, j = m - (m / NB) * NB;
    const int K = tile * 32 + lane;
    const int ne = a.ne;

    double out[4] = {0.0, 0.0, 0.0, 0.0};
    if (K < ne) {
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
            const double* c = a.icoef + (size_t)DG_ICOEF * a.inst[K];
            eps = c[0];
            alpha = c[1];
#pragma unroll
            for (int t = 0; t < 6; ++t) bc[t] = c[2 + t];
            sig_int = c[8];
            sig_bdry = c[9];
        }

        // ---- volume integrals ------------------------------------------------
        const double* vw = sm + L.vol_w;
        const double* vr = sm + L.vol_r;
        const double* vs = sm + L.vol_s;
        const double* vp = sm + L.vol_phi;
        const double* vdr = sm + L.vol_dr;
        const double* vds = sm + L.vol_ds;
        double acc = 0.0;
#pragma unroll 4
        for (int q = 0; q < QK; ++q) {
            const double w = vw[q] * det;
            const double pi = vp[q * NB + i], pj = vp[q * NB + j];
            const double dri = vdr[q * NB + i], dsi = vds[q * NB + i];
            const double drj = vdr[q * NB + j], dsj = vds[q * NB + j];
            const double gxi = i00 * dri + i10 * dsi, gyi = i01 * dri + i11 * dsi;
            const double gxj = i00 * drj + i10 * dsj, gyj = i01 * drj + i11 * dsj;
            const double x = x0 + j00 * vr[q] + j01 * vs[q];
            const double y = y0 + j10 * vr[q] + j11 * vs[q];
            const double bx = bc[0] + bc[1] * x + bc[2] * y;
            const double by = bc[3] + bc[4] * x + bc[5] * y;
            acc += w * (eps * (gxj * gxi + gyj * gyi) + (bx * gxj + by * gyj) * pi + alpha * pj * pi);
        }

        // ---- face integrals ----------------------------------------------------
        const double* fw = sm + L.face_w;
        const double* fr = sm + L.face_r;
        const double* fs = sm + L.face_s;
        const double* fp = sm + L.face_phi;
        const double* fdr = sm + L.face_dr;
        const double* fds = sm + L.face_ds;
        const double dV[3][2] = {{1.0, 0.0}, {-1.0, 1.0}, {0.0, -1.0}};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const int type = __ldg(a.ftype + (size_t)f * ne + K);
            const int Ln = __ldg(a.nbr + (size_t)f * ne + K);
            const int nf = __ldg(a.nface + (size_t)f * ne + K);
            const double tx = j00 * dV[f][0] + j01 * dV[f][1];
            const double ty = j10 * dV[f][0] + j11 * dV[f][1];
            const double len = sqrt(tx * tx + ty * ty);
            const double nx = ty / len, ny = -tx / len;
            const double he = len;  // h_e = |e|, b0 = 1
            double li00 = 0, li01 = 0, li10 = 0, li11 = 0;
            if (type == 0) {
                li00 = gload(a.geo, G_I00, ne, Ln);
                li01 = gload(a.geo, G_I01, ne, Ln);
                li10 = gload(a.geo, G_I10, ne, Ln);
                li11 = gload(a.geo, G_I11, ne, Ln);
            }
            const double sig = type == 0 ? sig_int : sig_bdry;
            double self = 0.0, cross = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double w = fw[q] * len;
                const int o = (f * NQ + q) * NB;
                const double pi = fp[o + i], pj = fp[o + j];
                const double gin = (i00 * fdr[o + i] + i10 * fds[o + i]) * nx + (i01 * fdr[o + i] + i11 * fds[o + i]) * ny;
                const double gjn = (i00 * fdr[o + j] + i10 * fds[o + j]) * nx + (i01 * fdr[o + j] + i11 * fds[o + j]) * ny;
                const double x = x0 + j00 * fr[f * NQ + q] + j01 * fs[f * NQ + q];
                const double y = y0 + j10 * fr[f * NQ + q] + j11 * fs[f * NQ + q];
                const double bn = (bc[0] + bc[1] * x + bc[2] * y) * nx + (bc[3] + bc[4] * x + bc[5] * y) * ny;
                const double up = bn < 0.0 ? bn : 0.0;
                if (type == 0) {
                    const int oo = (nf * NQ + (NQ - 1 - q)) * NB;   // same point seen from L
                    const double psj = fp[oo + j];
                    const double gpj = (li00 * fdr[oo + j] + li10 * fds[oo + j]) * nx +
                                       (li01 * fdr[oo + j] + li11 * fds[oo + j]) * ny;
                    self += w * (-0.5 * eps * gjn * pi + 0.5 * a.kappa * eps * gin * pj +
                                 sig * eps / he * pj * pi - up * pj * pi);
                    cross += w * (-0.5 * eps * gpj * pi - 0.5 * a.kappa * eps * gin * psj -
                                  sig * eps / he * psj * pi + up * psj * pi);
                } else if (type == 1) {
                    self += w * (-eps * gjn * pi + a.kappa * eps * gin * pj + sig * eps / he * pj * pi - up * pj * pi);
                } else {
                    self += w * (-up * pj * pi);
                }
            }
            acc += self;
            out[1 + f] = cross;
        }
        out[0] = acc;
    }
    // write entry m of the 4 blocks (zeros for padding lanes K >= ne)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (a.A64) a.A64[dg_blk_index<double>(K, s, m, NB, 4)] = out[s];
        if (a.A32) a.A32[dg_blk_index<float>(K, s, m, NB, 4)] = (float)out[s];
        if (a.A16) a.A16[dg_blk_index<__nv_bfloat16>(K, s, m, NB, 4)] = __double2bfloat16(out[s]);
    }
    // the last entry also clears the chunk padding after nb^2
    if (m == NB2 - 1) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (a.A64) for (int mm = NB2; mm < dg_chunks<double>(NB) * 2; ++mm) a.A64[dg_blk_index<double>(K, s, mm, NB, 4)] = 0.0;
            if (a.A32) for (int mm = NB2; mm < dg_chunks<float>(NB) * 4; ++mm) a.A32[dg_blk_index<float>(K, s, mm, NB, 4)] = 0.0f;
            if (a.A16) for (int mm = NB2; mm < dg_chunks<__nv_bfloat16>(NB) * 8; ++mm)
                a.A16[dg_blk_index<__nv_bfloat16>(K, s, mm, NB, 4)] = __double2bfloat16(0.0);
        }
    }
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
        const double he = len;
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
    const long warps_a = (long)h->ntiles * nb * nb;
    const long warps_r = (long)h->ntiles * nb;
    const unsigned ga = (unsigned)((warps_a + 7) / 8), gr = (unsigned)((warps_r + 7) / 8);
    switch (k) {
        case 1:
            k_assemble<1><<<ga, 256, smem, h->stream>>>(a);
            k_rhs<1><<<gr, 256, smem, h->stream>>>(a);
            break;
        case 2:
            k_assemble<2><<<ga, 256, smem, h->stream>>>(a);
            k_rhs<2><<<gr, 256, smem, h->stream>>>(a);
            break;
        case 3:
            k_assemble<3><<<ga, 256, smem, h->stream>>>(a);
            k_rhs<3><<<gr, 256, smem, h->stream>>>(a);
            break;
        default:
            return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

extern "C" dg_status dg_assemble(dg_handle* h, const dg_coeffs* c) {
    if (!h || !c) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    if (!(c->eps >= 0.0) || !(c->alpha == c->alpha)) return dg_fail(h, DG_ERR_INVALID_ARG, "eps must be >= 0");
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
    if ((s = dg_launch_assemble(h, c, kappa, sig, fac * sig)) != DG_OK) return s;
    h->assembled = true;
    h->asm_k = k;
    h->asm_store = h->p.store;
    h->mlp.coef[0] = c->eps;
    h->mlp.coef[1] = c->alpha;
    for (int t = 0; t < 6; ++t) h->mlp.coef[2 + t] = c->b[t];
    return DG_OK;
}
