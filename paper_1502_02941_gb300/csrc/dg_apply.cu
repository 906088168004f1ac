// dg_apply.cu -- the block-sparse operator apply y = Stiff x (the D u + C u +
// R u of Eq. (system)) and the block-Jacobi preconditioner.
//
// apply: one thread per element K, one warp per 32-element tile.  For each of
// the 4 slots the warp streams the slot's chunks as 32 x 16-byte loads
// (512 contiguous bytes per load instruction, evict-first so the blocks do not
// displace the vectors from L2), gathers the nb entries of x for the slot's
// element (K itself or its neighbour across face f) and accumulates the nb
// rows of y_K in registers.  Bytes per element: 4*nb^2*sizeof(TA) (fewer on the
// boundary) + 2*nb*sizeof(TX) + 12 (neighbour ids) -> HBM-bound.
#include "dg_kernels.cuh"

template <typename TV>
dg_status dg_mlp_correct(dg_handle* h, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz, const int* iuse);

// Gauss-Jordan inverse with partial pivoting (in f64) of each diagonal block
// A_KK read from the block copy of type TA; Binv64 may be NULL.
template <int NB, typename TA>
__global__ void __launch_bounds__(128) k_bj_setup(const TA* __restrict__ A, int ne, double* Binv64,
                                                   float* Binv32, int* flag) {
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    double M[NB][2 * NB];
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) {
            M[i][j] = (double)A[dg_blk_index<TA>(K, 0, i * NB + j, NB, 4)];
            M[i][NB + j] = i == j ? 1.0 : 0.0;
        }
    double amax = 0.0;
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) amax = fmax(amax, fabs(M[i][j]));
    bool singular = !(amax > 0.0) || !isfinite(amax);
    for (int c = 0; c < NB && !singular; ++c) {
        int p = c;
        for (int r = c + 1; r < NB; ++r)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (!(fabs(M[p][c]) > 1e-14 * amax)) {
            singular = true;
            break;
        }
        if (p != c)
            for (int j = 0; j < 2 * NB; ++j) {
                double t = M[c][j];
                M[c][j] = M[p][j];
                M[p][j] = t;
            }
        const double d = 1.0 / M[c][c];
        for (int j = 0; j < 2 * NB; ++j) M[c][j] *= d;
        for (int r = 0; r < NB; ++r) {
            if (r == c) continue;
            const double l = M[r][c];
            for (int j = 0; j < 2 * NB; ++j) M[r][j] -= l * M[c][j];
        }
    }
    if (singular) {
        atomicOr(flag, 1);
        for (int m = 0; m < NB * NB; ++m) {
            if (Binv64) Binv64[dg_blk_index<double>(K, 0, m, NB, 1)] = 0.0;
            Binv32[dg_blk_index<float>(K, 0, m, NB, 1)] = 0.0f;
        }
        return;
    }
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) {
            if (Binv64) Binv64[dg_blk_index<double>(K, 0, i * NB + j, NB, 1)] = M[i][NB + j];
            Binv32[dg_blk_index<float>(K, 0, i * NB + j, NB, 1)] = (float)M[i][NB + j];
        }
}

// Block (K, slot s) of A M^-1: A_{K,s} Binv_L with L the neighbour across face
// s-1, in f64; zero for a missing neighbour.  Slot 0, A_KK A_KK^-1 = I, is not
// formed: the applies of A M^-1 take it as the identity (k_apply, UNIT).  One
// thread per (element, slot); writes the f64 and / or f32 copy.
template <int NB>
__global__ void __launch_bounds__(128) k_ahat_setup(const double* __restrict__ A, const double* __restrict__ Binv,
                                                     const int* __restrict__ nbr, int ne, double* Ah64, float* Ah32) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4L * ne) return;
    const int K = (int)(t >> 2), s = (int)(t & 3);
    if (s == 0) return;
    const int L = __ldg(nbr + (size_t)(s - 1) * ne + K);
    double a[NB][NB], b[NB][NB];
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) {
            a[i][j] = L >= 0 ? A[dg_blk_index<double>(K, s, i * NB + j, NB, 4)] : 0.0;
            b[i][j] = L >= 0 ? Binv[dg_blk_index<double>(L, 0, i * NB + j, NB, 1)] : 0.0;
        }
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) {
            double c = 0.0;
            for (int l = 0; l < NB; ++l) c = fma(a[i][l], b[l][j], c);
            const int m = i * NB + j;
            if (Ah64) Ah64[dg_blk_index<double>(K, s, m, NB, 4)] = c;
            if (Ah32) Ah32[dg_blk_index<float>(K, s, m, NB, 4)] = (float)c;
        }
}

// A M^-1 for every stored precision (after the f64 inverses exist).  The
// arrays are cleared first, so chunk padding and padding lanes stay zero.
static dg_status ahat_setup(dg_handle* h) {
    const int nb = dg_nb(h->asm_k);
    const size_t per = (size_t)h->ntiles * 4 * 16 * 32;   // bytes per chunk row x chunks below
    // no bf16 copy: the bf16 inner solves keep block Jacobi on the bf16 blocks,
    // whose true residual they are checked against
    size_t need[2] = {0, 0};
    if (h->A64) need[0] = per * dg_chunks<double>(nb);
    if (h->A32) need[1] = per * dg_chunks<float>(nb);
    void** ptrs[2] = {(void**)&h->Ah64, (void**)&h->Ah32};
    dg_status s;
    for (int t = 0; t < 2; ++t) {
        if (need[t] != h->Ah_bytes[t]) {
            if ((s = dg_realloc(h, ptrs[t], need[t])) != DG_OK) return s;
            h->Ah_bytes[t] = need[t];
        }
        if (need[t]) DG_CK(h, cudaMemsetAsync(*ptrs[t], 0, need[t], h->stream));
    }
    const unsigned g = (unsigned)((4L * h->ne + 127) / 128);
    switch (nb) {
        case 3: k_ahat_setup<3><<<g, 128, 0, h->stream>>>(h->A64, h->Binv64, h->nbr, h->ne, h->Ah64, h->Ah32); break;
        case 6: k_ahat_setup<6><<<g, 128, 0, h->stream>>>(h->A64, h->Binv64, h->nbr, h->ne, h->Ah64, h->Ah32); break;
        case 10: k_ahat_setup<10><<<g, 128, 0, h->stream>>>(h->A64, h->Binv64, h->nbr, h->ne, h->Ah64, h->Ah32); break;
        default: return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

// Restricted additive Schwarz with one layer of overlap: for element K with
// face neighbours L_f, P = {K, L_f} and A_P the patch matrix (A's blocks
// between patch elements; neighbours couple only where they share a face).
// Row block K of A_P^-1 (NB x |P| NB) is stored in the 4 slots of K (slot 1+f
// multiplies r_{L_f}), so z = G r is one apply.  The rows come from solving
// A_P^T y_i = e_i (i over K's NB unknowns) by Gaussian elimination with
// partial pivoting in f64, one thread per element.
template <int NB>
__global__ void __launch_bounds__(64) k_ras_setup(const double* __restrict__ A, const int* __restrict__ nbr,
                                                   const int* __restrict__ nface, int ne, double* G64, float* G32,
                                                   int* flag) {
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    constexpr int NP = 4 * NB;
    double M[NP][NP + NB];
    int E[4], slotK[4], slotOf[4], cnt = 1;
    E[0] = K;
    slotOf[0] = 0;
    slotK[0] = 0;
    for (int f = 0; f < 3; ++f) {
        const int L = nbr[(size_t)f * ne + K];
        if (L >= 0) {
            E[cnt] = L;
            slotOf[cnt] = 1 + f;
            slotK[cnt] = 1 + nface[(size_t)f * ne + K];
            ++cnt;
        }
    }
    const int n = cnt * NB;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n + NB; ++b) M[a][b] = 0.0;
    // M = A_P^T | [e_0 .. e_{NB-1}]
    for (int p = 0; p < cnt; ++p)
        for (int q = 0; q < cnt; ++q) {
            int slot = -1;
            if (p == q) slot = 0;
            else if (p == 0) slot = slotOf[q];
            else if (q == 0) slot = slotK[p];
            else
                for (int f = 0; f < 3; ++f)
                    if (nbr[(size_t)f * ne + E[p]] == E[q]) slot = 1 + f;
            if (slot < 0) continue;
            for (int i = 0; i < NB; ++i)
                for (int j = 0; j < NB; ++j)
                    M[q * NB + j][p * NB + i] = A[dg_blk_index<double>(E[p], slot, i * NB + j, NB, 4)];
        }
    for (int i = 0; i < NB; ++i) M[i][n + i] = 1.0;
    double amax = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) amax = fmax(amax, fabs(M[a][b]));
    bool ok = amax > 0.0 && isfinite(amax);
    for (int c = 0; c < n && ok; ++c) {
        int pv = c;
        for (int a = c + 1; a < n; ++a)
            if (fabs(M[a][c]) > fabs(M[pv][c])) pv = a;
        if (!(fabs(M[pv][c]) > 1e-14 * amax)) {
            ok = false;
            break;
        }
        if (pv != c)
            for (int b = c; b < n + NB; ++b) {
                const double t = M[c][b];
                M[c][b] = M[pv][b];
                M[pv][b] = t;
            }
        const double inv = 1.0 / M[c][c];
        for (int a = c + 1; a < n; ++a) {
            const double l = M[a][c] * inv;
            if (l != 0.0)
                for (int b = c; b < n + NB; ++b) M[a][b] = fma(-l, M[c][b], M[a][b]);
        }
    }
    if (!ok) {
        atomicOr(flag, 2);
        return;
    }
    // back substitution for the NB right-hand sides (solutions overwrite them)
    for (int i = 0; i < NB; ++i)
        for (int a = n - 1; a >= 0; --a) {
            double t = M[a][n + i];
            for (int b = a + 1; b < n; ++b) t = fma(-M[a][b], M[b][n + i], t);
            M[a][n + i] = t / M[a][a];
        }
    // row i of K's block row: G_{K, slot(p)}[i][j] = y_i[p NB + j]
    for (int p = 0; p < cnt; ++p)
        for (int i = 0; i < NB; ++i)
            for (int j = 0; j < NB; ++j) {
                const double g = M[p * NB + j][n + i];
                const int m = i * NB + j;
                if (G64) G64[dg_blk_index<double>(K, slotOf[p], m, NB, 4)] = g;
                if (G32) G32[dg_blk_index<float>(K, slotOf[p], m, NB, 4)] = (float)g;
            }
}

static dg_status ras_setup(dg_handle* h) {
    const int nb = dg_nb(h->asm_k);
    const size_t per = (size_t)h->ntiles * 4 * 16 * 32;
    size_t need[2] = {per * dg_chunks<double>(nb), per * dg_chunks<float>(nb)};
    void** ptrs[2] = {(void**)&h->G64, (void**)&h->G32};
    dg_status s;
    for (int t = 0; t < 2; ++t) {
        if (need[t] != h->G_bytes[t]) {
            if ((s = dg_realloc(h, ptrs[t], need[t])) != DG_OK) return s;
            h->G_bytes[t] = need[t];
        }
        DG_CK(h, cudaMemsetAsync(*ptrs[t], 0, need[t], h->stream));
    }
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    const unsigned g = (unsigned)((h->ne + 63) / 64);
    switch (nb) {
        case 3: k_ras_setup<3><<<g, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, h->ne, h->G64, h->G32, h->dflag); break;
        case 6: k_ras_setup<6><<<g, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, h->ne, h->G64, h->G32, h->dflag); break;
        case 10: k_ras_setup<10><<<g, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, h->ne, h->G64, h->G32, h->dflag); break;
        default: return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    int flag = 0;
    DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flag) return dg_fail(h, DG_ERR_SINGULAR_BLOCK, "a patch matrix is singular");
    return DG_OK;
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int NB>
static dg_status apply_nb(dg_handle* h, int dtype, const void* x, void* y) {
    const ElemShape es = elem_shape(h);
    switch (dtype) {
        case DG_F64:
            if (!h->A64) return dg_fail(h, DG_ERR_STATE, "f64 blocks not stored");
            k_apply<NB, double, double, double><<<es.grid, es.block, 0, h->stream>>>(
                h->A64, h->nbr, (const double*)x, (double*)y, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());
            break;
        case DG_F32:
            if (!h->A32) return dg_fail(h, DG_ERR_STATE, "f32 blocks not stored");
            k_apply<NB, float, float, float><<<es.grid, es.block, 0, h->stream>>>(
                h->A32, h->nbr, (const float*)x, (float*)y, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());
            break;
        case DG_BF16:
            if (!h->A16) return dg_fail(h, DG_ERR_STATE, "bf16 blocks not stored");
            k_apply<NB, __nv_bfloat16, float, float><<<es.grid, es.block, 0, h->stream>>>(
                h->A16, h->nbr, (const float*)x, (float*)y, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());
            break;
        default:
            return dg_fail(h, DG_ERR_INVALID_ARG, "dtype");
    }
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

dg_status dg_launch_apply(dg_handle* h, int dtype, const void* x, void* y) {
    switch (dg_nb(h->asm_k)) {
        case 3: return apply_nb<3>(h, dtype, x, y);
        case 6: return apply_nb<6>(h, dtype, x, y);
        case 10: return apply_nb<10>(h, dtype, x, y);
    }
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

extern "C" dg_status dg_apply(dg_handle* h, int dtype, const void* x, void* y) {
    if (!h || !x || !y) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (x == y) return dg_fail(h, DG_ERR_INVALID_ARG, "x and y must not overlap");
    if (!dg_aligned16(x) || !dg_aligned16(y)) return dg_fail(h, DG_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    return dg_launch_apply(h, dtype, x, y);
}

template <int NB>
static dg_status bj_apply_nb(dg_handle* h, int dtype, const void* r, void* z) {
    const unsigned grid = (unsigned)((h->ne + 255) / 256);
    if (dtype == DG_F64)
        k_bj_apply<NB, double, double, double><<<grid, 256, 0, h->stream>>>(
            h->Binv64, (const double*)r, (double*)z, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());
    else
        k_bj_apply<NB, float, float, float><<<grid, 256, 0, h->stream>>>(
            h->Binv32, (const float*)r, (float*)z, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

dg_status dg_launch_bj_apply(dg_handle* h, int dtype, const void* r, void* z, const double* scale) {
    (void)scale;
    switch (dg_nb(h->asm_k)) {
        case 3: return bj_apply_nb<3>(h, dtype, r, z);
        case 6: return bj_apply_nb<6>(h, dtype, r, z);
        case 10: return bj_apply_nb<10>(h, dtype, r, z);
    }
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

dg_status dg_launch_bj_setup(dg_handle* h) {
    const int nb = dg_nb(h->asm_k);
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "block Jacobi needs the f64 blocks (DG_STORE_F64)");
    dg_status s;
    size_t b64 = (size_t)h->ntiles * dg_chunks<double>(nb) * 512;
    size_t b32 = (size_t)h->ntiles * dg_chunks<float>(nb) * 512;
    if ((s = dg_ensure(h, (void**)&h->Binv64, &h->cap_binv64, b64)) != DG_OK) return s;
    if ((s = dg_ensure(h, (void**)&h->Binv32, &h->cap_binv32, b32)) != DG_OK) return s;
    DG_CK(h, cudaMemsetAsync(h->Binv64, 0, b64, h->stream));
    DG_CK(h, cudaMemsetAsync(h->Binv32, 0, b32, h->stream));
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    const unsigned grid = (unsigned)((h->ne + 127) / 128);
    // with a bf16 copy stored, the bf16 inner solves get the inverses of the
    // bf16 diagonal blocks themselves (M^-1 A_bf16 has identity diagonal blocks)
    float* B16 = nullptr;
    if (h->A16) {
        if ((s = dg_ensure(h, (void**)&h->Binv16, &h->cap_binv16, b32)) != DG_OK) return s;
        DG_CK(h, cudaMemsetAsync(h->Binv16, 0, b32, h->stream));
        B16 = h->Binv16;
    }
    switch (nb) {
        case 3:
            k_bj_setup<3, double><<<grid, 128, 0, h->stream>>>(h->A64, h->ne, h->Binv64, h->Binv32, h->dflag);
            if (B16) k_bj_setup<3, __nv_bfloat16><<<grid, 128, 0, h->stream>>>(h->A16, h->ne, nullptr, B16, h->dflag);
            break;
        case 6:
            k_bj_setup<6, double><<<grid, 128, 0, h->stream>>>(h->A64, h->ne, h->Binv64, h->Binv32, h->dflag);
            if (B16) k_bj_setup<6, __nv_bfloat16><<<grid, 128, 0, h->stream>>>(h->A16, h->ne, nullptr, B16, h->dflag);
            break;
        case 10:
            k_bj_setup<10, double><<<grid, 128, 0, h->stream>>>(h->A64, h->ne, h->Binv64, h->Binv32, h->dflag);
            if (B16) k_bj_setup<10, __nv_bfloat16><<<grid, 128, 0, h->stream>>>(h->A16, h->ne, nullptr, B16, h->dflag);
            break;
        default: return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += B16 ? 2 : 1;
    DG_LAUNCH_CK(h);
    int flag = 0;
    DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flag) return dg_fail(h, DG_ERR_SINGULAR_BLOCK, "a diagonal block is singular");
    return ahat_setup(h);
}

extern "C" dg_status dg_precond_setup(dg_handle* h, int kind) {
    DG_WS_SCOPE(h, DG_WS_PRECOND);
    if (!h) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (kind == DG_PRECOND_NONE) return DG_OK;
    if (kind != DG_PRECOND_BLOCK_JACOBI && kind != DG_PRECOND_MLP && kind != DG_PRECOND_SCHWARZ)
        return dg_fail(h, DG_ERR_INVALID_ARG, "precond kind");
    if (kind == DG_PRECOND_MLP && (!h->mlp.packed || h->mlp.nb != dg_nb(h->asm_k)))
        return dg_fail(h, DG_ERR_STATE, "MLP preconditioner: dg_mlp_init / dg_mlp_set_weights for this degree first");
    h->bj_ok = false;
    h->ras_ok = false;
    dg_status s = dg_launch_bj_setup(h);
    if (s == DG_OK) h->bj_ok = true;
    if (s == DG_OK && kind == DG_PRECOND_SCHWARZ) {
        if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the Schwarz preconditioner needs the f64 blocks");
        s = ras_setup(h);
        if (s == DG_OK) h->ras_ok = true;
    }
    return s;
}

extern "C" dg_status dg_precond_apply(dg_handle* h, int dtype, const void* r, void* z) {
    if (!h || !r || !z) return DG_ERR_INVALID_ARG;
    if (!h->bj_ok) return dg_fail(h, DG_ERR_STATE, "preconditioner not set up");
    if (!dg_aligned16(r) || !dg_aligned16(z)) return dg_fail(h, DG_ERR_INVALID_ARG, "r and z must be 16-byte aligned");
    if (dtype != DG_F64 && dtype != DG_F32 && dtype != DG_BF16) return dg_fail(h, DG_ERR_INVALID_ARG, "dtype");
    if (h->p.precond == DG_PRECOND_SCHWARZ) {
        if (!h->ras_ok) return dg_fail(h, DG_ERR_STATE, "Schwarz preconditioner not set up");
        const unsigned grid = (unsigned)((h->ne + 255) / 256);
        const int nb = dg_nb(h->asm_k);
#define DG_RAS_APPLY(NBV)                                                                                         \
        if (nb == NBV) {                                                                                          \
            if (dtype == DG_F64)                                                                                  \
                k_apply<NBV, double, double, double><<<grid, 256, 0, h->stream>>>(                                \
                    h->G64, h->nbr, (const double*)r, (double*)z, h->ne, dctl_none(), vsel_fixed(), vsel_fixed()); \
            else                                                                                                  \
                k_apply<NBV, float, float, float><<<grid, 256, 0, h->stream>>>(                                   \
                    h->G32, h->nbr, (const float*)r, (float*)z, h->ne, dctl_none(), vsel_fixed(), vsel_fixed());  \
        }
        DG_RAS_APPLY(3)
        DG_RAS_APPLY(6)
        DG_RAS_APPLY(10)
#undef DG_RAS_APPLY
        h->nlaunch += 1;
        DG_LAUNCH_CK(h);
        return DG_OK;
    }
    dg_status s = dg_launch_bj_apply(h, dtype == DG_F64 ? DG_F64 : DG_F32, r, z, nullptr);
    if (s != DG_OK || h->p.precond != DG_PRECOND_MLP || !h->mlp.packed) return s;
    const int one = 1;
    DG_CK(h, cudaMemcpyAsync(h->mlp.on, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (dtype == DG_F64)
        return dg_mlp_correct<double>(h, (const double*)r, (double*)z, dctl_none(), vsel_fixed(), vsel_fixed(), nullptr);
    return dg_mlp_correct<float>(h, (const float*)r, (float*)z, dctl_none(), vsel_fixed(), vsel_fixed(), nullptr);
}
