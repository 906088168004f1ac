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

// Dense LU with partial pivoting, blocked and right-looking, on the row-major
// n x n matrix M in global memory: P M = L U with the unit lower L below the
// diagonal and U on and above it; b is permuted with the rows.  Each panel of
// bw <= LU_B columns is factored in shared memory (k_lu_panel), its row swaps
// are applied to the other columns and U12 = L11^-1 A12 is formed
// (k_lu_swap_trsm), and A22 -= L21 U12 (k_lu_gemm).  The kernels are launched
// programmatically dependent on their predecessor (each waits for it before
// touching memory).
//
// Widest panel: 16 columns.  The panel's rank-1 updates (about R bw^2 / 2
// FMAs per panel) run on one SM, whose FP64 pipe does two FMAs a clock on this
// GPU; the trailing update takes the rest of the GPU.
#define LU_B 16
#define LU_SMEM (216 * 1024)   // shared memory of the panel kernel
#define LU_PERM (2 * LU_B)     // rows a panel's swaps can touch

// Panel width for R = n - k0 remaining rows: the largest power of two <= LU_B
// whose column-major panel (column stride R | 1) fits in LU_SMEM.
static int lu_panel_width(int R) {
    int bw = LU_B;
    while (bw > 1 && (size_t)(R | 1) * bw * sizeof(double) > LU_SMEM) bw >>= 1;
    return bw;
}

// Block argmax of (|value|, row) pairs, the lowest row on ties; every thread
// gets the winner.  One pair per warp is staged in sv / si.
__device__ __forceinline__ void lu_argmax(double& best, int& bi, double* sv, int* si) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[wid] = best; si[wid] = bi; }
    __syncthreads();
    best = lane < nw ? sv[lane] : -1.0;
    bi = lane < nw ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
}

// Factor the panel of columns [k0, k0 + bw) over rows k0..n-1 in shared memory
// (one CTA, a multiple of 32 threads): per column the pivot (largest |entry|,
// lowest row on ties), the swap of the two rows within the panel, the
// multipliers below the diagonal and the rank-1 update of the panel's later
// columns, which also finds the next column's pivot candidates.  Then the
// panel's swaps, in order, composed into one permutation of the rows they touch:
// perm = {count, rows[LU_PERM], src[LU_PERM]}, row rows[q] receiving the content
// of row src[q]; b is permuted with it.  A zero pivot sets *flag (the factors
// are then meaningless; no access leaves M).
__global__ void __launch_bounds__(1024) k_lu_panel(double* M, double* b, int* perm, int n, int k0, int bw,
                                                   int* flag) {
    dg_grid_release();
    dg_grid_wait();
    extern __shared__ double P[];   // P[j * Rp + i] = M[k0 + i][k0 + j]
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int sp[LU_B];
    __shared__ int prow[LU_PERM], psrc[LU_PERM];
    __shared__ int pcount;
    const int R = n - k0, Rp = R | 1;
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < R * bw; e += nt) {
        const int i = e / bw, j = e - i * bw;
        P[j * Rp + i] = M[(long)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = t; i < R; i += nt) {
        const double v = fabs(P[i]);
        if (v > best) { best = v; bi = i; }
    }
    for (int c = 0; c < bw; ++c) {
        lu_argmax(best, bi, sv, si);
        // no candidate wins when the column holds only NaNs: keep row c
        const int p = (bi >= c && bi < R) ? bi : c;
        if (t == 0) {
            sp[c] = p;
            if (!(best > 0.0)) *flag = 1;
        }
        if (p != c && t < bw) {
            const double a = P[t * Rp + c];
            P[t * Rp + c] = P[t * Rp + p];
            P[t * Rp + p] = a;
        }
        __syncthreads();
        const double d = P[c * Rp + c];
        const double inv = d != 0.0 ? 1.0 / d : 0.0;
        best = -1.0;
        bi = 0x7fffffff;
        for (int i = c + 1 + t; i < R; i += nt) {
            const double l = P[c * Rp + i] * inv;
            P[c * Rp + i] = l;
            for (int j = c + 1; j < bw; ++j) P[j * Rp + i] = fma(-l, P[j * Rp + c], P[j * Rp + i]);
            if (c + 1 < bw) {
                const double v = fabs(P[(c + 1) * Rp + i]);
                if (v > best) { best = v; bi = i; }
            }
        }
    }
    if (t == 0) {   // compose the swaps (local row indices)
        int cnt = 0;
        for (int c = 0; c < bw; ++c) {
            const int r1 = c, r2 = sp[c];
            if (r1 == r2) continue;
            int q1 = -1, q2 = -1;
            for (int q = 0; q < cnt; ++q) {
                if (prow[q] == r1) q1 = q;
                if (prow[q] == r2) q2 = q;
            }
            if (q1 < 0) { q1 = cnt; prow[cnt] = r1; psrc[cnt] = r1; ++cnt; }
            if (q2 < 0) { q2 = cnt; prow[cnt] = r2; psrc[cnt] = r2; ++cnt; }
            const int a = psrc[q1];
            psrc[q1] = psrc[q2];
            psrc[q2] = a;
        }
        pcount = cnt;
        perm[0] = cnt;
        for (int q = 0; q < cnt; ++q) {
            perm[1 + q] = k0 + prow[q];
            perm[1 + LU_PERM + q] = k0 + psrc[q];
        }
    }
    __syncthreads();
    for (int e = t; e < R * bw; e += nt) {
        const int i = e / bw, j = e - i * bw;
        M[(long)(k0 + i) * n + k0 + j] = P[j * Rp + i];
    }
    const int cnt = pcount;
    double bv = 0.0;
    if (t < cnt) bv = b[k0 + psrc[t]];
    __syncthreads();
    if (t < cnt) b[k0 + prow[t]] = bv;
}

// The panel's row permutation on every column outside it (one thread per
// column: all the touched entries loaded, then stored), then U12 = L11^-1 A12
// on the columns right of it (unit lower L11 staged in shared memory).  One
// warp per block, so that the FP64 work of the triangular solves spreads over
// many SMs.
__global__ void __launch_bounds__(32) k_lu_swap_trsm(double* M, const int* perm, int n, int k0, int bw) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ double L[LU_B][LU_B + 1];
    __shared__ int prow[LU_PERM], psrc[LU_PERM];
    const int t = threadIdx.x;
    for (int e = t; e < bw * bw; e += blockDim.x) {
        const int i = e / bw, l = e - i * bw;
        L[i][l] = M[(long)(k0 + i) * n + k0 + l];
    }
    const int cnt = perm[0];
    for (int q = t; q < cnt; q += blockDim.x) {
        prow[q] = perm[1 + q];
        psrc[q] = perm[1 + LU_PERM + q];
    }
    __syncthreads();
    const int q0 = blockIdx.x * blockDim.x + t;   // over the n - bw columns outside the panel
    if (q0 >= n - bw) return;
    const int j = q0 < k0 ? q0 : q0 + bw;
    double v[LU_PERM];
#pragma unroll
    for (int q = 0; q < LU_PERM; ++q)
        if (q < cnt) v[q] = M[(long)psrc[q] * n + j];
#pragma unroll
    for (int q = 0; q < LU_PERM; ++q)
        if (q < cnt) M[(long)prow[q] * n + j] = v[q];
    if (j < k0 + bw) return;
    double u[LU_B];
#pragma unroll
    for (int i = 0; i < LU_B; ++i) u[i] = i < bw ? M[(long)(k0 + i) * n + j] : 0.0;
#pragma unroll
    for (int i = 1; i < LU_B; ++i) {
        if (i < bw) {
            double s = u[i];
#pragma unroll
            for (int l = 0; l < i; ++l) s = fma(-L[i][l], u[l], s);
            u[i] = s;
        }
    }
#pragma unroll
    for (int i = 1; i < LU_B; ++i)
        if (i < bw) M[(long)(k0 + i) * n + j] = u[i];
}

// A22 -= L21 U12 over rows and columns k0+bw..n-1 (inner dimension bw <=
// LU_B): 32 x 32 output tiles, 256 threads with 4 outputs each, the tile's L21
// rows and U12 columns staged in shared memory.
__global__ void __launch_bounds__(256) k_lu_gemm(double* M, int n, int k0, int bw) {
    dg_grid_release();
    dg_grid_wait();
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

// L y = b (unit lower), then U x = y, in blocks of 32 rows with b in shared
// memory (n <= 4096); x overwrites b.  Per block, warp 0 solves the diagonal
// block (lane = row, the solved entries passed by shuffles), then one warp per
// remaining row subtracts the block's contribution (lane = column: coalesced
// 256-byte reads of M).
__global__ void __launch_bounds__(1024) k_lu_trisolve(const double* M, double* b, int n) {
    dg_grid_release();
    dg_grid_wait();
    extern __shared__ double sb[];
    __shared__ double D[32][33];
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5, nw = nt >> 5;
    for (int i = t; i < n; i += nt) sb[i] = b[i];
    for (int j0 = 0; j0 < n; j0 += 32) {   // forward
        const int w = min(32, n - j0);
        for (int e = t; e < w * w; e += nt) D[e / w][e % w] = M[(long)(j0 + e / w) * n + j0 + e % w];
        __syncthreads();
        if (wid == 0) {
            double y = lane < w ? sb[j0 + lane] : 0.0;
            for (int c = 0; c < w - 1; ++c) {
                const double yc = __shfl_sync(0xffffffffu, y, c);
                if (lane > c && lane < w) y = fma(-D[lane][c], yc, y);
            }
            if (lane < w) sb[j0 + lane] = y;
        }
        __syncthreads();
        const double yl = lane < w ? sb[j0 + lane] : 0.0;
        for (int i = j0 + w + wid; i < n; i += nw) {
            double v = lane < w ? M[(long)i * n + j0 + lane] * yl : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sb[i] -= v;
        }
        __syncthreads();
    }
    for (int j1 = n; j1 > 0; j1 -= 32) {   // backward
        const int j0 = max(0, j1 - 32), w = j1 - j0;
        for (int e = t; e < w * w; e += nt) D[e / w][e % w] = M[(long)(j0 + e / w) * n + j0 + e % w];
        __syncthreads();
        if (wid == 0) {
            double y = lane < w ? sb[j0 + lane] : 0.0;
            for (int c = w - 1; c >= 0; --c) {
                if (lane == c) y = y / D[c][c];
                const double xc = __shfl_sync(0xffffffffu, y, c);
                if (lane < c) y = fma(-D[lane][c], xc, y);
            }
            if (lane < w) sb[j0 + lane] = y;
        }
        __syncthreads();
        const double xl = lane < w ? sb[j0 + lane] : 0.0;
        for (int i = wid; i < j0; i += nw) {
            double v = lane < w ? M[(long)i * n + j0 + lane] * xl : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sb[i] -= v;
        }
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
    const size_t mbytes = (sizeof(double) * (size_t)n * n + 255) / 256 * 256;
    dg_status s = dg_scratch(h, mbytes + sizeof(int) * (1 + 2 * LU_PERM));
    if (s != DG_OK) return s;
    double* M = h->scratch;
    int* perm = reinterpret_cast<int*>(reinterpret_cast<char*>(h->scratch) + mbytes);
    DG_CK(h, cudaMemsetAsync(M, 0, sizeof(double) * (size_t)n * n, h->stream));
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    long tot = (long)h->ne * 4 * nb * nb;
    k_densify<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(h->A64, h->nbr, h->ne, nb, M, n);
    DG_CK(h, cudaMemcpyAsync(x, F ? F : h->F, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    DG_CK(h, cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, LU_SMEM));
    DG_CK(h, cudaFuncSetAttribute(k_lu_trisolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * n)));
    const bool pdl = h->pdl && h->stream != nullptr;
    const int nn = (int)n;
    int launches = 1;
    for (int k0 = 0; k0 < nn;) {
        const int R = nn - k0;
        const int bw = std::min(lu_panel_width(R), R);
        // about four rows a thread: fewer warps make the per-column barriers cheaper
        const int nt = std::min(1024, std::max(32, ((R + 3) / 4 + 31) / 32 * 32));
        const size_t sm = sizeof(double) * (size_t)(R | 1) * bw;
        dg_launch_smem(h, pdl, sm, k_lu_panel, dim3(1), dim3(nt), M, x, perm, nn, k0, bw, h->dflag);
        ++launches;
        if (nn > bw) {
            dg_launch(h, pdl, k_lu_swap_trsm, dim3((unsigned)((nn - bw + 31) / 32)), dim3(32), M, (const int*)perm,
                      nn, k0, bw);
            ++launches;
        }
        const int rest = R - bw;
        if (rest > 0) {
            const unsigned gt = (unsigned)((rest + 31) / 32);
            dg_launch(h, pdl, k_lu_gemm, dim3(gt, gt), dim3(256), M, nn, k0, bw);
            ++launches;
        }
        k0 += bw;
    }
    dg_launch_smem(h, pdl, sizeof(double) * n, k_lu_trisolve, dim3(1), dim3(1024), (const double*)M, x, nn);
    h->nlaunch += launches + 1;
    DG_LAUNCH_CK(h);
    int flag = 0;
    DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flag) return dg_fail(h, DG_ERR_SINGULAR_BLOCK, "singular matrix in the dense solve");
    return DG_OK;
}
