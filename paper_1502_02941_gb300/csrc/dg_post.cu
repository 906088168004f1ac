// dg_post.cu -- the paper's dg_error (L2 error and h_max, Sec. 2.4), point
// evaluation of u_h, and the direct solve Stiff\F (Sec. 2.3) for small systems.
#include <math.h>
#include <string.h>

#include <vector>

#include "dg_internal.cuh"

// ---------------------------------------------------------------------------
// L2 error: sum_K sum_q w_q detJ (u_h(x_q) - u(x_q))^2, then a second pass.
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(256) k_l2(const double* __restrict__ x, const double* __restrict__ uex,
                                             const double* __restrict__ geo, const double* __restrict__ tab,
                                             TabLayout L, int ne, double* partials) {
    extern __shared__ double sm[];
    const int qe = L.qerr;
    for (int t = threadIdx.x; t < qe * (NB + 1); t += blockDim.x)
        sm[t] = t < qe ? tab[L.err_w + t] : tab[L.err_phi + t - qe];
    __syncthreads();
    __shared__ double sh[32];
    double acc = 0.0;
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
        double c[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) c[i] = x[(size_t)K * NB + i];
        const double det = geo[G_DET * (size_t)ne + K];
        double e = 0.0;
        for (int q = 0; q < qe; ++q) {
            double u = 0.0;
#pragma unroll
            for (int i = 0; i < NB; ++i) u += c[i] * sm[qe + q * NB + i];
            const double d = u - uex[(size_t)K * qe + q];
            e += sm[q] * d * d;
        }
        acc += e * det;
    }
    acc = dg_block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_sum_partials(const double* p, int n, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    s = dg_block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

extern "C" dg_status dg_l2_error(dg_handle* h, const double* x, const double* uex_q, double* l2, double* hmax) {
    if (!h || !x || !uex_q) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    DG_CK(h, cudaSetDevice(h->device));
    const int k = h->p.degree;
    dg_status s = dg_ensure_tables(h, k);
    if (s != DG_OK) return s;
    const int G = 1024;
    if ((s = dg_scratch(h, sizeof(double) * (G + 1))) != DG_OK) return s;
    double* part = h->scratch;
    const size_t smem = sizeof(double) * h->tl.qerr * (dg_nb(k) + 1);
    switch (k) {
        case 1: k_l2<3><<<G, 256, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
        case 2: k_l2<6><<<G, 256, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
        case 3: k_l2<10><<<G, 256, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
    }
    k_sum_partials<<<1, 1024, 0, h->stream>>>(part, G, part + G);
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    double e2 = 0.0;
    DG_CK(h, cudaMemcpyAsync(&e2, part + G, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (l2) *l2 = sqrt(e2);
    if (hmax) *hmax = h->hmax;
    return DG_OK;
}

// ---------------------------------------------------------------------------
// point evaluation
// ---------------------------------------------------------------------------
__global__ void k_eval(const double* __restrict__ x, const double* __restrict__ phi, int nb, int np, int ne,
                       double* out) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long)ne * np) return;
    int K = (int)(g / np), p = (int)(g - (long)K * np);
    double u = 0.0;
    for (int i = 0; i < nb; ++i) u += x[(size_t)K * nb + i] * phi[p * nb + i];
    out[g] = u;
}

extern "C" dg_status dg_eval(dg_handle* h, const double* x, int np, const double* rs, double* out) {
    if (!h || !x || !rs || !out || np < 1 || np > 4096) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    DG_CK(h, cudaSetDevice(h->device));
    const int k = h->p.degree, nb = dg_nb(k);
    std::vector<double> phi((size_t)np * nb);
    for (int p = 0; p < np; ++p) {
        const double r = rs[2 * p], s = rs[2 * p + 1];
        if (!(r >= -1e-12 && s >= -1e-12 && r + s <= 1.0 + 1e-12 && s < 1.0))
            return dg_fail(h, DG_ERR_INVALID_ARG, "reference point outside the triangle (or at the top vertex)");
        dg_dubiner(k, r, s, phi.data() + (size_t)p * nb, nullptr, nullptr);
    }
    dg_status st = dg_scratch(h, sizeof(double) * phi.size());
    if (st != DG_OK) return st;
    DG_CK(h, cudaMemcpyAsync(h->scratch, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice, h->stream));
    long n = (long)h->ne * np;
    k_eval<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(x, h->scratch, nb, np, h->ne, out);
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    // the staging buffer is reused by later calls: make the copy complete first
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

// ---------------------------------------------------------------------------
// dense direct solve (small systems)
// ---------------------------------------------------------------------------
__global__ void k_densify(const double* __restrict__ A, const int* __restrict__ nbr, int ne, int nb, double* M,
                          long n) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = 4L * nb * nb;
    if (g >= (long)ne * per) return;
    int K = (int)(g / per);
    int rem = (int)(g - (long)K * per);
    int s = rem / (nb * nb), m = rem - s * nb * nb;
    int i = m / nb, j = m - i * nb;
    int L = s == 0 ? K : nbr[(size_t)(s - 1) * ne + K];
    if (L < 0) return;
    M[((long)K * nb + i) * n + (long)L * nb + j] = A[dg_blk_index<double>(K, s, m, nb, 4)];
}

// Dense LU with partial pivoting, blocked and right-looking (panels of LU_B
// columns), on the row-major n x n matrix M in global memory; the row swaps
// are applied to whole rows of M and to b, so that at the end P M = L U with
// the unit lower L below the diagonal, U on and above it, and b = P b.
#define LU_B 32

// Factor the panel of columns [k0, k0 + bw) over rows k0..n-1 (one CTA):
// per column the pivot (largest |M[r][c]|, lowest index on ties), the swap of
// rows c and p across all n columns and in b, the multipliers below the
// diagonal, and the rank-1 update of the panel's remaining columns.  A zero
// pivot sets *flag (the factors are then meaningless; no access leaves M).
__global__ void __launch_bounds__(1024) k_lu_panel(double* M, double* b, int n, int k0, int bw, int* flag) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int piv;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5;
    for (int c = k0; c < k0 + bw; ++c) {
        double best = -1.0;
        int bi = c;
        for (int r = c + t; r < n; r += nt) {
            const double v = fabs(M[(long)r * n + c]);
            if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sv[wid] = best; si[wid] = bi; }
        __syncthreads();
        if (t == 0) {
            double bb = -1.0;
            int ii = c;
            for (int w = 0; w < nt / 32; ++w)
                if (sv[w] > bb || (sv[w] == bb && si[w] < ii)) { bb = sv[w]; ii = si[w]; }
            piv = ii;
            if (!(bb > 0.0)) *flag = 1;
        }
        __syncthreads();
        const int p = piv;
        if (p != c) {
            for (int j = t; j < n; j += nt) {
                const double a = M[(long)c * n + j];
                M[(long)c * n + j] = M[(long)p * n + j];
                M[(long)p * n + j] = a;
            }
            if (t == 0) {
                const double a = b[c];
                b[c] = b[p];
                b[p] = a;
            }
        }
        __syncthreads();
        const double d = M[(long)c * n + c];
        const double inv = d != 0.0 ? 1.0 / d : 0.0;
        for (int r = c + 1 + t; r < n; r += nt) M[(long)r * n + c] *= inv;
        __syncthreads();
        const int w = k0 + bw - c - 1;   // panel columns right of c
        if (w > 0) {
            const long cnt = (long)(n - c - 1) * w;
            for (long e = t; e < cnt; e += nt) {
                const int r = c + 1 + (int)(e / w), j = c + 1 + (int)(e % w);
                M[(long)r * n + j] -= M[(long)r * n + c] * M[(long)c * n + j];
            }
        }
        __syncthreads();
    }
}

// U12 = L11^-1 A12: rows k0..k0+bw-1, columns k0+bw..n-1, unit lower L11; one
// thread per column.
__global__ void __launch_bounds__(256) k_lu_trsm(double* M, int n, int k0, int bw) {
    const int j = k0 + bw + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int i = 1; i < bw; ++i) {
        double s = M[(long)(k0 + i) * n + j];
        for (int l = 0; l < i; ++l) s -= M[(long)(k0 + i) * n + k0 + l] * M[(long)(k0 + l) * n + j];
        M[(long)(k0 + i) * n + j] = s;
    }
}

// A22 -= L21 U12 over rows and columns k0+bw..n-1 (inner dimension bw <=
// LU_B): 32 x 32 output tiles, 256 threads with 4 outputs each, the tile's L21
// rows and U12 columns staged in shared memory.
__global__ void __launch_bounds__(256) k_lu_gemm(double* M, int n, int k0, int bw) {
    __shared__ double Ls[32][LU_B + 1], Us[LU_B][32 + 1];
    const int r0 = k0 + bw + blockIdx.y * 32, c0 = k0 + bw + blockIdx.x * 32;
    const int t = threadIdx.x;
    for (int e = t; e < 32 * LU_B; e += 256) {
        const int rr = e / LU_B, kk = e % LU_B;
        Ls[rr][kk] = (r0 + rr < n && kk < bw) ? M[(long)(r0 + rr) * n + k0 + kk] : 0.0;
        const int k2 = e / 32, cc = e % 32;
        Us[k2][cc] = (c0 + cc < n && k2 < bw) ? M[(long)(k0 + k2) * n + c0 + cc] : 0.0;
    }
    __syncthreads();
    const int cc = t & 31, rq = t >> 5;   // rows rq, rq + 8, rq + 16, rq + 24
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < bw; ++k) {
        const double u = Us[k][cc];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(Ls[rq + 8 * q][k], u, acc[q]);
    }
    if (c0 + cc >= n) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + rq + 8 * q;
        if (r < n) M[(long)r * n + c0 + cc] -= acc[q];
    }
}

// L y = b (unit lower), then U x = y, column-oriented with b in shared memory
// (n <= 4096); x overwrites b.
__global__ void __launch_bounds__(1024) k_lu_trisolve(const double* M, double* b, int n) {
    extern __shared__ double sb[];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < n; i += nt) sb[i] = b[i];
    __syncthreads();
    for (int j = 0; j < n; ++j) {          // forward: b_i -= L_ij y_j, i > j
        const double yj = sb[j];
        for (int i = j + 1 + t; i < n; i += nt) sb[i] -= M[(long)i * n + j] * yj;
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {     // backward: x_j = y_j / U_jj, then b_i -= U_ij x_j, i < j
        const double xj = sb[j] / M[(long)j * n + j];
        __syncthreads();
        if (t == 0) sb[j] = xj;
        for (int i = t; i < j; i += nt) sb[i] -= M[(long)i * n + j] * xj;
        __syncthreads();
    }
    for (int i = t; i < n; i += nt) b[i] = sb[i];
}

extern "C" dg_status dg_dense_solve(dg_handle* h, const double* F, double* x) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    if (!h->assembled || !h->A64) return dg_fail(h, DG_ERR_STATE, "not assembled with f64 blocks");
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->asm_k);
    const long n = (long)h->ne * nb;
    if (n > 4096) return dg_fail(h, DG_ERR_INVALID_ARG, "dense solve is limited to 4096 unknowns");
    dg_status s = dg_scratch(h, sizeof(double) * (size_t)n * n + 64);
    if (s != DG_OK) return s;
    double* M = h->scratch;
    DG_CK(h, cudaMemsetAsync(M, 0, sizeof(double) * (size_t)n * n, h->stream));
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    long tot = (long)h->ne * 4 * nb * nb;
    k_densify<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(h->A64, h->nbr, h->ne, nb, M, n);
    DG_CK(h, cudaMemcpyAsync(x, F ? F : h->F, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    const int nn = (int)n;
    int launches = 1;
    for (int k0 = 0; k0 < nn; k0 += LU_B) {
        const int bw = nn - k0 < LU_B ? nn - k0 : LU_B;
        k_lu_panel<<<1, 1024, 0, h->stream>>>(M, x, nn, k0, bw, h->dflag);
        ++launches;
        const int rest = nn - k0 - bw;
        if (rest > 0) {
            k_lu_trsm<<<(unsigned)((rest + 255) / 256), 256, 0, h->stream>>>(M, nn, k0, bw);
            const unsigned gt = (unsigned)((rest + 31) / 32);
            k_lu_gemm<<<dim3(gt, gt), 256, 0, h->stream>>>(M, nn, k0, bw);
            launches += 2;
        }
    }
    DG_CK(h, cudaFuncSetAttribute(k_lu_trisolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * n)));
    k_lu_trisolve<<<1, 1024, sizeof(double) * n, h->stream>>>(M, x, nn);
    h->nlaunch += launches + 1;
    DG_LAUNCH_CK(h);
    int flag = 0;
    DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flag) return dg_fail(h, DG_ERR_SINGULAR_BLOCK, "singular matrix in the dense solve");
    return DG_OK;
}
