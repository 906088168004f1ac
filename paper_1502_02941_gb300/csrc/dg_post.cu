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
template <typename T>
__global__ void k_densify(const double* __restrict__ A, const int* __restrict__ nbr, int ne, int nb, T* M, long n) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = 4L * nb * nb;
    if (g >= (long)ne * per) return;
    int K = (int)(g / per);
    int rem = (int)(g - (long)K * per);
    int s = rem / (nb * nb), m = rem - s * nb * nb;
    int i = m / nb, j = m - i * nb;
    int L = s == 0 ? K : nbr[(size_t)(s - 1) * ne + K];
    if (L < 0) return;
    M[((long)K * nb + i) * n + (long)L * nb + j] = (T)A[dg_blk_index<double>(K, s, m, nb, 4)];
}

// Dense LU with partial pivoting, blocked and right-looking, on the row-major
// n x n matrix M (f64 or f32) in global memory: P M = L U with the unit lower L
// below the diagonal and U on and above it.  Each panel of bw columns is
// factored in shared memory (k_lu_panel), its row swaps are applied to the
// other columns and U12 = L11^-1 A12 is formed (k_lu_swap_trsm), and
// A22 -= L21 U12 (k_lu_gemm).  Each panel's swaps are kept, composed into one
// permutation, for the solves.  The kernels are launched programmatically
// dependent on their predecessor (each waits for it before touching memory).
//
// The dense solve factors in f32 and refines in f64 (LU-based iterative
// refinement): this GPU's FP32 pipe is 64x its FP64 pipe, and the panel's
// dependent per-column steps are latency-bound on one SM, where FP64
// operations are long.  Each refinement step solves with the f32 factors for
// the correction of the f64 residual F - A x (the f64 block operator), so x
// converges to f64 accuracy when cond(A) u_f32 << 1; otherwise, or on a zero
// f32 pivot, the f64 factorization runs instead.  Panel width: up to 32
// columns in f32, 16 in f64 (where the panel's rank-1 updates, about
// R bw^2 / 2 FMAs, run on one SM's FP64 pipe, two FMAs a clock).
#define LU_BMAX 32
#define LU_SMEM (216 * 1024)    // shared memory of the panel kernel
#define LU_PERM (2 * LU_BMAX)   // rows a panel's swaps can touch
#define LU_PREC (1 + 2 * LU_PERM)   // ints per recorded panel permutation
#define LU_IR_MAX 10            // refinement steps before the f64 fallback

template <typename T>
static int lu_panel_width(int R) {
    int bw = sizeof(T) == 4 ? 32 : 16;
    while (bw > 1 && (size_t)(R | 1) * bw * sizeof(T) > LU_SMEM) bw >>= 1;
    return bw;
}

// Copy of the panel between M (row-major) and P (column-major, column stride
// Rp), eight accesses in flight per thread.
template <typename T, bool TO_SMEM>
__device__ __forceinline__ void lu_panel_copy(T* M, T* P, int n, int k0, int R, int Rp, int bw) {
    const int t = threadIdx.x, nt = blockDim.x, tot = R * bw;
    for (int e0 = t; e0 < tot; e0 += 8 * nt) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nt;
            if (e < tot) {
                const int i = e / bw, j = e - i * bw;
                v[u] = TO_SMEM ? M[(long)(k0 + i) * n + k0 + j] : P[j * Rp + i];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nt;
            if (e < tot) {
                const int i = e / bw, j = e - i * bw;
                if (TO_SMEM) P[j * Rp + i] = v[u];
                else M[(long)(k0 + i) * n + k0 + j] = v[u];
            }
        }
    }
}

// The off-panel work of a panel CTA (all its threads): the panel's row
// permutation (rows k0 + prow[q] receive rows k0 + psrc[q]) on every column
// outside it, one thread per column with all touched entries loaded before any
// is stored; then right of the panel U12 = L11^-1 A12, the unit lower L11's
// entry (r, l) read at L11[r * sr + l * sl].  (The row indices are read through volatile so that the
// 2 x cnt of them are not hoisted out of the column loop into registers.)
template <typename T, int UB>
__device__ __forceinline__ void lu_panel_offpanel(T* M, int n, int k0, int bw, int cnt, const volatile int* vsrc,
                                               const volatile int* vrow, const T* L11, int sr, int sl) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int q0 = t; q0 < n - bw; q0 += nt) {
        const int j = q0 < k0 ? q0 : q0 + bw;
        T w[2 * UB];
#pragma unroll
        for (int q = 0; q < 2 * UB; ++q)
            if (q < cnt) w[q] = M[(long)(k0 + vsrc[q]) * n + j];
#pragma unroll
        for (int q = 0; q < 2 * UB; ++q)
            if (q < cnt) M[(long)(k0 + vrow[q]) * n + j] = w[q];
    }
    __syncthreads();   // the permuted rows, stored by other threads, are read below
    for (int j = k0 + bw + t; j < n; j += nt) {
        T uu[UB];
#pragma unroll
        for (int r = 0; r < UB; ++r) uu[r] = r < bw ? M[(long)(k0 + r) * n + j] : (T)0;
#pragma unroll
        for (int l = 0; l < UB - 1; ++l) {
            if (l + 1 < bw) {
#pragma unroll
                for (int r = l + 1; r < UB; ++r)
                    if (r < bw) uu[r] = fma(-L11[r * sr + l * sl], uu[l], uu[r]);
            }
        }
#pragma unroll
        for (int r = 1; r < UB; ++r)
            if (r < bw) M[(long)(k0 + r) * n + j] = uu[r];
    }
}

// The same out of line (the f64 register-row panel kernel spills with it inlined).
template <typename T, int UB>
__device__ __noinline__ void lu_panel_offpanel_call(T* M, int n, int k0, int bw, int cnt, const volatile int* vsrc,
                                                    const volatile int* vrow, const T* L11, int sr, int sl) {
    lu_panel_offpanel<T, UB>(M, n, k0, bw, cnt, vsrc, vrow, L11, sr, sl);
}

// Warp argmax of (|value|, row) pairs, the lowest row on ties; every lane
// gets the winner.
template <typename T>
__device__ __forceinline__ void lu_warp_argmax(T& best, int& bi) {
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
}

// Factor the panel of columns [k0, k0 + bw) (bw <= 32) over rows k0..n-1 in
// shared memory (one CTA of nw <= 16 warps; lane = panel column, warp w takes
// the rows c+1+w, c+1+w+nw, ... of each column step c).  Per column: the pivot
// (largest |entry|, lowest row on ties) from the per-warp candidates, the swap
// of the two rows within the panel, then per row the multiplier (one broadcast
// load) and the rank-1 update of the row's later columns (one FMA per lane);
// lane c+1 of each warp tracks the next column's candidates on the way.  Then
// the panel's swaps, in order, composed into one permutation of the rows they
// touch: perm = {count, rows[LU_PERM], src[LU_PERM]}, row rows[q] receiving
// the content of row src[q].  With trsm set the same CTA then applies that
// permutation to every column outside the panel and forms U12 = L11^-1 A12
// (else k_lu_swap_trsm does).  A zero (or NaN) pivot sets *flag (the factors
// are then meaningless; no access leaves M).
#define LU_PANEL_THREADS 512
template <typename T>
__global__ void __launch_bounds__(LU_PANEL_THREADS) k_lu_panel(T* M, int* perm, int n, int k0, int bw, int trsm,
                                                               int* flag) {
    dg_grid_release();
    dg_grid_wait();
    extern __shared__ __align__(16) unsigned char lu_smem[];
    T* P = reinterpret_cast<T*>(lu_smem);   // P[j * Rp + i] = M[k0 + i][k0 + j]
    __shared__ T sv[16];
    __shared__ int si[16];
    __shared__ int sp[LU_BMAX];
    __shared__ int prow[LU_PERM], psrc[LU_PERM];
    __shared__ int pcount;
    const int R = n - k0, Rp = R | 1;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5, nw = nt >> 5;
    lu_panel_copy<T, true>(M, P, n, k0, R, Rp, bw);
    __syncthreads();
    {   // candidates of column 0, one per warp
        T best = (T)-1;
        int bi = 0x7fffffff;
        for (int i = t; i < R; i += nt) {
            const T v = fabs(P[i]);
            if (v > best) { best = v; bi = i; }
        }
        lu_warp_argmax<T>(best, bi);
        if (lane == 0) { sv[wid] = best; si[wid] = bi; }
    }
    for (int c = 0; c < bw; ++c) {
        __syncthreads();   // candidates written, previous updates done
        T best = lane < nw ? sv[lane] : (T)-1;
        int bi = lane < nw ? si[lane] : 0x7fffffff;
        lu_warp_argmax<T>(best, bi);
        // no candidate wins when the column holds only NaNs: keep row c
        const int p = (bi >= c && bi < R) ? bi : c;
        if (t == 0) {
            sp[c] = p;
            if (!(best > (T)0) || !isfinite(best)) *flag = 1;
        }
        if (wid == 0 && p != c && lane < bw) {
            const T a = P[lane * Rp + c];
            P[lane * Rp + c] = P[lane * Rp + p];
            P[lane * Rp + p] = a;
        }
        __syncthreads();
        const T d = P[c * Rp + c];
        const T inv = d != (T)0 ? (T)1 / d : (T)0;
        const bool act = lane > c && lane < bw;
        const T u = act ? P[lane * Rp + c] : (T)0;
        T cb = (T)-1;   // next column's candidate (meaningful in lane c + 1)
        int ci = 0x7fffffff;
        int i = c + 1 + wid;
        for (; i + 3 * nw < R; i += 4 * nw) {   // four rows at a time
            T x[4], y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = P[c * Rp + i + q * nw];
#pragma unroll
            for (int q = 0; q < 4; ++q) y[q] = act ? P[lane * Rp + i + q * nw] : (T)0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x[q] *= inv;
                y[q] = fma(-x[q], u, y[q]);
            }
            __syncwarp();   // every lane has read the multipliers before lane c overwrites them
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (act) P[lane * Rp + i + q * nw] = y[q];
                else if (lane == c) P[c * Rp + i + q * nw] = x[q];
                const T a = fabs(y[q]);
                if (a > cb) { cb = a; ci = i + q * nw; }
            }
        }
        for (; i < R; i += nw) {
            const T l = P[c * Rp + i] * inv;
            const T y = act ? fma(-l, u, P[lane * Rp + i]) : (T)0;
            __syncwarp();
            if (act) P[lane * Rp + i] = y;
            else if (lane == c) P[c * Rp + i] = l;
            const T a = fabs(y);
            if (a > cb) { cb = a; ci = i; }
        }
        if (c + 1 < bw && lane == c + 1) { sv[wid] = cb; si[wid] = ci; }
    }
    __syncthreads();
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
    lu_panel_copy<T, false>(M, P, n, k0, R, Rp, bw);
    if (!trsm) return;
    constexpr int UB = sizeof(T) == 4 ? LU_BMAX : LU_BMAX / 2;   // widest panel of type T
    lu_panel_offpanel<T, UB>(M, n, k0, bw, pcount, psrc, prow, P, 1, Rp);   // L11 (r, l) = P[l * Rp + r]
}

// The same panel factorization for R <= LU_PANEL_THREADS rows with each row in
// the registers of one thread (local row t in thread t) for the whole panel:
// the column loop is unrolled, so every entry index is a constant.  Pivoting is
// lazy: rows stay in their threads, the winner of column c (the largest |entry|
// among the rows not yet chosen, lowest original row on ties, which is the row
// partial pivoting with row swaps picks) broadcasts its row through shared
// memory, and the rows not yet chosen update from it; every thread follows its
// row's position through the equivalent sequence of row swaps (all threads see
// each swap), and at the end every row is stored at its position.  Results, permutation record and the
// optional off-panel work as k_lu_panel.
template <typename T, int BW>
__global__ void __launch_bounds__(LU_PANEL_THREADS) k_lu_panel_reg(T* M, int* perm, int n, int k0, int bw, int trsm,
                                                                   int* flag) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ T sv[16];
    __shared__ int si[16];
    __shared__ T xr[BW];           // the pivot row of a column step
    __shared__ T L11[BW][BW + 1];
    __shared__ int sp[BW];
    __shared__ int prow[2 * BW], psrc[2 * BW];
    __shared__ int pcount;
    const int R = n - k0;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const bool mine = t < R;
    bool open = mine;   // not chosen as a pivot yet
    int mypos = t;      // the row's position under the swaps so far
    T v[BW];
#pragma unroll
    for (int j = 0; j < BW; ++j) v[j] = (mine && j < bw) ? M[(long)(k0 + t) * n + k0 + j] : (T)0;
    // ties go to the lowest current position, as in the swapping algorithm
#pragma unroll
    for (int c = 0; c < BW; ++c) {
        if (c >= bw) break;   // block-uniform
        __syncthreads();      // positions and the previous pivot row are settled
        T best = open ? fabs(v[c]) : (T)-1;
        int bi = open ? mypos : 0x7fffffff;
        lu_warp_argmax<T>(best, bi);
        if (lane == 0) { sv[wid] = best; si[wid] = bi; }
        __syncthreads();
        best = lane < nw ? sv[lane] : (T)-1;
        bi = lane < nw ? si[lane] : 0x7fffffff;
        lu_warp_argmax<T>(best, bi);
        // no candidate wins when the column holds only NaNs: keep position c
        const int q = (bi >= c && bi < R) ? bi : c;   // the pivot's position (position c is open)
        if (open && mypos == q) {
            open = false;
#pragma unroll
            for (int j = 0; j < BW; ++j) xr[j] = v[j];
        }
        mypos = mypos == q ? c : (mypos == c ? q : mypos);   // the swap of positions c and q
        if (t == 0) {
            sp[c] = q;
            if (!(best > (T)0) || !isfinite(best)) *flag = 1;
        }
        __syncthreads();
        const T d = xr[c];
        const T inv = d != (T)0 ? (T)1 / d : (T)0;
        if (open) {
            const T l = v[c] * inv;
            v[c] = l;
#pragma unroll
            for (int j = c + 1; j < BW; ++j) v[j] = fma(-l, xr[j], v[j]);
        }
    }
    const int me = mypos;
#pragma unroll
    for (int j = 0; j < BW; ++j)
        if (mine && j < bw) M[(long)(k0 + me) * n + k0 + j] = v[j];
    if (mine && me < bw) {
#pragma unroll
        for (int j = 0; j < BW; ++j) L11[me][j] = v[j];
    }
    __syncthreads();
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
    if (!trsm) return;
    if constexpr (sizeof(T) == 8)
        lu_panel_offpanel_call<T, BW>(M, n, k0, bw, pcount, psrc, prow, &L11[0][0], BW + 1, 1);
    else
        lu_panel_offpanel<T, BW>(M, n, k0, bw, pcount, psrc, prow, &L11[0][0], BW + 1, 1);
}

// The panel's row permutation on every column outside it (one thread per
// column: all the touched entries loaded, then stored), then U12 = L11^-1 A12
// on the columns right of it (unit lower L11 staged in shared memory).  One
// warp per block, so that the work of the triangular solves spreads over many
// SMs.
template <typename T>
__global__ void __launch_bounds__(32) k_lu_swap_trsm(T* M, const int* perm, int n, int k0, int bw) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ T L[LU_BMAX][LU_BMAX + 1];
    __shared__ int prow[LU_PERM], psrc[LU_PERM];
    const int t = threadIdx.x;
    for (int e0 = t; e0 < bw * bw; e0 += 8 * blockDim.x) {   // eight loads in flight
        T lv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < bw * bw) lv[u] = M[(long)(k0 + e / bw) * n + k0 + e % bw];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < bw * bw) L[e / bw][e % bw] = lv[u];
        }
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
    constexpr int UB = sizeof(T) == 4 ? LU_BMAX : LU_BMAX / 2;   // widest panel of type T
    T v[2 * UB];
#pragma unroll
    for (int q = 0; q < 2 * UB; ++q)
        if (q < cnt) v[q] = M[(long)psrc[q] * n + j];
#pragma unroll
    for (int q = 0; q < 2 * UB; ++q)
        if (q < cnt) M[(long)prow[q] * n + j] = v[q];
    if (j < k0 + bw) return;
    T u[UB];
#pragma unroll
    for (int i = 0; i < UB; ++i) u[i] = i < bw ? M[(long)(k0 + i) * n + j] : (T)0;
    // column-oriented forward substitution: the updates of one level are independent
#pragma unroll
    for (int l = 0; l < UB - 1; ++l) {
        if (l + 1 < bw) {
#pragma unroll
            for (int i = l + 1; i < UB; ++i)
                if (i < bw) u[i] = fma(-L[i][l], u[l], u[i]);
        }
    }
#pragma unroll
    for (int i = 1; i < UB; ++i)
        if (i < bw) M[(long)(k0 + i) * n + j] = u[i];
}

// A22 -= L21 U12 over rows and columns k0+bw..n-1 (inner dimension bw <=
// LU_BMAX): 32 x 32 output tiles, 256 threads with 4 outputs each, the tile's
// L21 rows and U12 columns staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_lu_gemm(T* M, int n, int k0, int bw) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ T Ls[32][LU_BMAX + 1], Us[LU_BMAX][32 + 1];
    const int r0 = k0 + bw + blockIdx.y * 32, c0 = k0 + bw + blockIdx.x * 32;
    const int t = threadIdx.x;
    for (int e = t; e < 32 * LU_BMAX; e += 256) {
        const int rr = e / LU_BMAX, kk = e % LU_BMAX;
        Ls[rr][kk] = (r0 + rr < n && kk < bw) ? M[(long)(r0 + rr) * n + k0 + kk] : (T)0;
        const int k2 = e / 32, cc = e % 32;
        Us[k2][cc] = (c0 + cc < n && k2 < bw) ? M[(long)(k0 + k2) * n + c0 + cc] : (T)0;
    }
    __syncthreads();
    const int cc = t & 31, rq = t >> 5;   // rows rq, rq + 8, rq + 16, rq + 24
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
    for (int k = 0; k < bw; ++k) {
        const T u = Us[k][cc];
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

// Inverses of the 32 x 32 diagonal blocks of the factors (one warp per block,
// the last one ragged): Dinv[b] holds L_bb^-1 (unit lower) and then U_bb^-1,
// each stored transposed (entry (i, c) at c * 32 + i, zero outside the
// block), so that a solve applies a diagonal block as one coalesced
// matrix-vector product.  Lane k computes column k of each inverse by forward
// (backward) substitution.
template <typename T>
__global__ void __launch_bounds__(32) k_lu_diag_inv(const T* __restrict__ M, int n, T* __restrict__ Dinv) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ T D[32][33], X[32][33];
    const int lane = threadIdx.x, j0 = blockIdx.x * 32, w = min(32, n - j0);
    for (int r = 0; r < 32; ++r) D[r][lane] = (r < w && lane < w) ? M[(long)(j0 + r) * n + j0 + lane] : (T)0;
    __syncwarp();
    T* out = Dinv + (size_t)blockIdx.x * 2048;
    for (int i = 0; i < 32; ++i) {   // L^-1: X[m][lane] = 0 for m < lane
        T acc = i == lane ? (T)1 : (T)0;
        for (int m = lane; m < i; ++m) acc = fma(-D[i][m], X[m][lane], acc);
        X[i][lane] = (i < w && lane < w) ? acc : (T)0;
    }
    __syncwarp();
    for (int c = 0; c < 32; ++c) out[c * 32 + lane] = X[lane][c];
    __syncwarp();
    for (int i = 31; i >= 0; --i) {   // U^-1: X[m][lane] = 0 for m > lane
        T acc = i == lane ? (T)1 : (T)0;
        for (int m = i + 1; m <= lane; ++m) acc = fma(-D[i][m], X[m][lane], acc);
        X[i][lane] = (i <= lane && lane < w) ? acc / D[i][i] : (T)0;
    }
    __syncwarp();
    for (int c = 0; c < 32; ++c) out[1024 + c * 32 + lane] = X[lane][c];
}

// One solve with the factors (one CTA, b in shared memory, n <= 4096): the
// recorded panel permutations applied to b in order, L y = P b (unit lower),
// then U z = y, in blocks of 32 rows.  Per block, warp 0 applies the inverse of
// the diagonal block (k_lu_diag_inv; lane = row, coalesced reads), then one
// thread per remaining row subtracts the block's contribution (its 32 entries
// of M loaded together).  With acc set x += z in f64, otherwise x = z;
// norms[0] = max |z_i| and norms[1] = max |x_i| (after the update).  b is read
// in f64 and rounded to T; b and x may be the same vector.
template <typename T>
__device__ __forceinline__ T lu_row_block(const T* __restrict__ Mrow, const T* y, int w, bool vec) {
    T v[32];
    if (vec && w == 32) {   // 16-byte aligned row: eight (f32) or sixteen (f64) vector loads
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 a = reinterpret_cast<const float4*>(Mrow)[q];
                v[4 * q] = a.x;
                v[4 * q + 1] = a.y;
                v[4 * q + 2] = a.z;
                v[4 * q + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const double2 a = reinterpret_cast<const double2*>(Mrow)[q];
                v[2 * q] = a.x;
                v[2 * q + 1] = a.y;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = c < w ? Mrow[c] : (T)0;
    }
    T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
        a0 = fma(v[c], y[c], a0);
        a1 = fma(v[c + 1], y[c + 1], a1);
        a2 = fma(v[c + 2], y[c + 2], a2);
        a3 = fma(v[c + 3], y[c + 3], a3);
    }
    return (a0 + a1) + (a2 + a3);
}

#define LU_SOLVE_THREADS 512   // 128 registers a thread: the 32 row entries stay in registers
template <typename T>
__global__ void __launch_bounds__(LU_SOLVE_THREADS) k_lu_solve(const T* __restrict__ M, const T* __restrict__ Dinv,
                                                               const int* __restrict__ perms, int npanel,
                                                               const double* b, double* x, int n, int acc,
                                                               double* norms) {
    dg_grid_release();
    dg_grid_wait();
    extern __shared__ __align__(16) unsigned char lu_smem[];
    T* sb = reinterpret_cast<T*>(lu_smem);
    __shared__ T yb[32];
    __shared__ double red[64];
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5, nw = nt >> 5;
    for (int i = t; i < n; i += nt) sb[i] = (T)b[i];
    __syncthreads();
    for (int pnl = 0; pnl < npanel; ++pnl) {   // the row swaps, panel by panel
        const int* pp = perms + (size_t)pnl * LU_PREC;
        const int cnt = pp[0];
        T v = (T)0;
        if (t < cnt) v = sb[pp[1 + LU_PERM + t]];
        __syncthreads();
        if (t < cnt) sb[pp[1 + t]] = v;
        __syncthreads();
    }
    // rows of M start 16-byte aligned when n is a multiple of 16 / sizeof(T)
    const bool vec = (n % (16 / (int)sizeof(T))) == 0;
    T li[32];   // warp 0: the current diagonal block's inverse, column `lane` (prefetched)
    if (wid == 0)
#pragma unroll
        for (int c = 0; c < 32; ++c) li[c] = Dinv[c * 32 + lane];
    for (int j0 = 0; j0 < n; j0 += 32) {   // forward
        const int w = min(32, n - j0);
        if (wid == 0) {
            T y = (T)0;
#pragma unroll
            for (int c = 0; c < 32; ++c) y = fma(li[c], c < w ? sb[j0 + c] : (T)0, y);
            yb[lane] = y;   // zero for lane >= w
            __syncwarp();
            if (lane < w) sb[j0 + lane] = y;
        }
        __syncthreads();
        if (wid == 0) {   // the next block's inverse (forward), else the last block's U^-1
            const T* nx = j0 + 32 < n ? Dinv + (size_t)(j0 / 32 + 1) * 2048 : Dinv + (size_t)(j0 / 32) * 2048 + 1024;
#pragma unroll
            for (int c = 0; c < 32; ++c) li[c] = nx[c * 32 + lane];
        }
        for (int i = j0 + w + t; i < n; i += nt) sb[i] -= lu_row_block(M + (long)i * n + j0, yb, w, vec);
        __syncthreads();
    }
    for (int j0 = (n - 1) / 32 * 32; j0 >= 0; j0 -= 32) {   // backward, the diagonal blocks of the forward pass
        const int w = min(32, n - j0);
        if (wid == 0) {
            T y = (T)0;
#pragma unroll
            for (int c = 0; c < 32; ++c) y = fma(li[c], c < w ? sb[j0 + c] : (T)0, y);
            yb[lane] = y;
            __syncwarp();
            if (lane < w) sb[j0 + lane] = y;
        }
        __syncthreads();
        if (wid == 0 && j0 > 0) {   // the previous block's U^-1
            const T* nx = Dinv + (size_t)(j0 / 32 - 1) * 2048 + 1024;
#pragma unroll
            for (int c = 0; c < 32; ++c) li[c] = nx[c * 32 + lane];
        }
        for (int i = t; i < j0; i += nt) sb[i] -= lu_row_block(M + (long)i * n + j0, yb, w, vec);
        __syncthreads();
    }
    double mz = 0.0, mx = 0.0;
    for (int i = t; i < n; i += nt) {
        const double z = (double)sb[i];
        const double xi = acc ? x[i] + z : z;
        x[i] = xi;
        mz = fmax(mz, fabs(z));
        mx = fmax(mx, fabs(xi));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mz = fmax(mz, __shfl_xor_sync(0xffffffffu, mz, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { red[wid] = mz; red[32 + wid] = mx; }
    __syncthreads();
    if (t == 0) {
        for (int q = 1; q < nw; ++q) { mz = fmax(mz, red[q]); mx = fmax(mx, red[32 + q]); }
        norms[0] = mz;
        norms[1] = mx;
    }
}

// r = F - AX and norms[2] = max |r_i| (one CTA, n <= 4096); a non-finite
// entry makes norms[2] infinite.
__global__ void __launch_bounds__(1024) k_lu_resid(const double* __restrict__ F, const double* __restrict__ AX,
                                                   double* __restrict__ r, int n, double* norms) {
    dg_grid_release();
    dg_grid_wait();
    __shared__ double red[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = F[i] - AX[i];
        r[i] = v;
        m = isfinite(v) ? fmax(m, fabs(v)) : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
        norms[2] = m;
    }
}

// norms[3] = max_i sum_j |M_ij| (the infinity norm of the dense matrix; one
// warp per row, the maximum over non-negative floats taken on their bits).
template <typename T>
__global__ void k_lu_anorm(const T* __restrict__ M, int n, unsigned int* bits) {
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    float s = 0.f;
    for (int j = lane; j < n; j += 32) s += fabsf((float)M[(long)i * n + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicMax(bits, __float_as_uint(s));
}
__global__ void k_lu_anorm_fin(const unsigned int* bits, double* norms) { norms[3] = (double)__uint_as_float(*bits); }

// The factorization of the dense n x n matrix M of type T; the panel
// permutations go to perms (LU_PREC ints per panel).  Returns the panel count.
template <typename T>
static int lu_factor(dg_handle* h, T* M, int* perms, int nn, bool pdl, int* launches) {
    int npanel = 0;
    for (int k0 = 0; k0 < nn; ++npanel) {
        const int R = nn - k0;
        const int bw = std::min(lu_panel_width<T>(R), R);
        // one warp per 32 rows, at most 16 warps
        const int nt = std::min(LU_PANEL_THREADS, (R + 31) / 32 * 32);
        const size_t sm = sizeof(T) * (size_t)(R | 1) * bw;
        int* perm = perms + (size_t)npanel * LU_PREC;
        // up to 1024 unknowns the panel CTA also swaps the other columns and forms
        // U12 (two columns a thread at most); beyond, a kernel over many SMs does
        const int trsm = nn <= 1024 ? 1 : 0;
        if (R <= LU_PANEL_THREADS)   // a row per thread, in registers; eight warps at least for the off-panel work
            dg_launch(h, pdl, k_lu_panel_reg<T, sizeof(T) == 4 ? 32 : 16>, dim3(1), dim3(std::max(nt, 256)), M, perm,
                      nn, k0, bw, trsm, h->dflag);
        else
            dg_launch_smem(h, pdl, sm, k_lu_panel<T>, dim3(1), dim3(nt), M, perm, nn, k0, bw, trsm, h->dflag);
        ++*launches;
        if (nn > bw && !trsm) {
            dg_launch(h, pdl, k_lu_swap_trsm<T>, dim3((unsigned)((nn - bw + 31) / 32)), dim3(32), M,
                      (const int*)perm, nn, k0, bw);
            ++*launches;
        }
        const int rest = R - bw;
        if (rest > 0) {
            const unsigned gt = (unsigned)((rest + 31) / 32);
            dg_launch(h, pdl, k_lu_gemm<T>, dim3(gt, gt), dim3(256), M, nn, k0, bw);
            ++*launches;
        }
        k0 += bw;
    }
    return npanel;
}

// Upper bound on the panel count of an n x n factorization of type T.
template <typename T>
static int lu_max_panels(int nn) {
    int np = 0;
    for (int k0 = 0; k0 < nn; ++np) k0 += std::min(lu_panel_width<T>(nn - k0), nn - k0);
    return np;
}

extern "C" dg_status dg_dense_solve(dg_handle* h, const double* F, double* x) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    if (!h->assembled || !h->A64) return dg_fail(h, DG_ERR_STATE, "not assembled with f64 blocks");
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->asm_k);
    const long n = (long)h->ne * nb;
    if (n > 4096) return dg_fail(h, DG_ERR_INVALID_ARG, "dense solve is limited to 4096 unknowns");
    const int nn = (int)n;
    // scratch: the matrix (f64 size, used as f32 first), the panel permutations,
    // the diagonal-block inverses, F, the residual and A x (f64), norms and a
    // bit word
    const size_t mbytes = (sizeof(double) * (size_t)n * n + 255) / 256 * 256;
    const int maxp = std::max(lu_max_panels<float>(nn), lu_max_panels<double>(nn));
    const size_t pbytes = (sizeof(int) * (size_t)maxp * LU_PREC + 255) / 256 * 256;
    const int nbk = (nn + 31) / 32;
    const size_t ibytes = sizeof(double) * 2048 * (size_t)nbk;
    const size_t vbytes = (sizeof(double) * (size_t)n + 255) / 256 * 256;
    dg_status s = dg_scratch(h, mbytes + pbytes + ibytes + 3 * vbytes + 8 * sizeof(double));
    if (s != DG_OK) return s;
    char* base = reinterpret_cast<char*>(h->scratch);
    int* perms = reinterpret_cast<int*>(base + mbytes);
    void* dinv = base + mbytes + pbytes;
    char* vb = base + mbytes + pbytes + ibytes;
    double* Fv = reinterpret_cast<double*>(vb);
    double* r = reinterpret_cast<double*>(vb + vbytes);
    double* ax = reinterpret_cast<double*>(vb + 2 * vbytes);
    double* norms = reinterpret_cast<double*>(vb + 3 * vbytes);
    unsigned int* bits = reinterpret_cast<unsigned int*>(norms + 4);
    double hn[4];
    const bool pdl = h->pdl && h->stream != nullptr;
    const long tot = (long)h->ne * 4 * nb * nb;
    const unsigned gdn = (unsigned)((tot + 255) / 256);
    int launches = 0;
    DG_CK(h, cudaFuncSetAttribute(k_lu_panel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, LU_SMEM));
    DG_CK(h, cudaFuncSetAttribute(k_lu_panel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, LU_SMEM));
    DG_CK(h, cudaFuncSetAttribute(k_lu_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * n)));
    DG_CK(h, cudaMemcpyAsync(Fv, F ? F : h->F, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    // f32 factorization and f64 refinement: stop when the residual is at the
    // level of f64 rounding, ||r|| <= sqrt(n) eps ||A|| ||x|| (infinity norms)
    if (!h->dense_f64) {
        float* M = reinterpret_cast<float*>(h->scratch);
        DG_CK(h, cudaMemsetAsync(M, 0, sizeof(float) * (size_t)n * n, h->stream));
        DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
        DG_CK(h, cudaMemsetAsync(bits, 0, sizeof(unsigned int), h->stream));
        k_densify<float><<<gdn, 256, 0, h->stream>>>(h->A64, h->nbr, h->ne, nb, M, n);
        k_lu_anorm<float><<<(unsigned)((nn + 7) / 8), 256, 0, h->stream>>>(M, nn, bits);
        k_lu_anorm_fin<<<1, 1, 0, h->stream>>>(bits, norms);
        launches += 3;
        const int np = lu_factor<float>(h, M, perms, nn, pdl, &launches);
        float* Di = reinterpret_cast<float*>(dinv);
        dg_launch(h, pdl, k_lu_diag_inv<float>, dim3(nbk), dim3(32), (const float*)M, nn, Di);
        dg_launch_smem(h, pdl, sizeof(float) * n, k_lu_solve<float>, dim3(1), dim3(LU_SOLVE_THREADS), (const float*)M,
                       (const float*)Di, (const int*)perms, np, (const double*)Fv, x, nn, 0, norms);   // x = LU^-1 F
        launches += 2;
        int flag = 0;
        DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
        double prev = INFINITY;
        for (int it = 0; flag == 0 && it <= LU_IR_MAX; ++it) {
            s = dg_launch_apply(h, DG_F64, x, ax);   // r = F - A x
            if (s != DG_OK) return s;
            dg_launch(h, pdl, k_lu_resid, dim3(1), dim3(1024), (const double*)Fv, (const double*)ax, r, nn, norms);
            launches += 2;
            DG_CK(h, cudaMemcpyAsync(hn, norms, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            DG_CK(h, cudaStreamSynchronize(h->stream));
            if (!isfinite(hn[2]) || !isfinite(hn[1])) break;
            if (hn[2] <= sqrt((double)n) * 2.220446049250313e-16 * hn[3] * hn[1]) {
                h->nlaunch += launches;
                DG_LAUNCH_CK(h);
                return DG_OK;
            }
            if (it == LU_IR_MAX || (it >= 2 && hn[2] > 0.5 * prev)) break;   // out of steps, or not contracting
            prev = hn[2];
            dg_launch_smem(h, pdl, sizeof(float) * n, k_lu_solve<float>, dim3(1), dim3(LU_SOLVE_THREADS),
                           (const float*)M, (const float*)Di, (const int*)perms, np, (const double*)r, x, nn, 1,
                           norms);   // x += LU^-1 r
            ++launches;
        }
    }
    // f64 factorization (the f32 one met a zero pivot, or refinement did not converge)
    double* M = reinterpret_cast<double*>(h->scratch);
    DG_CK(h, cudaMemsetAsync(M, 0, sizeof(double) * (size_t)n * n, h->stream));
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    k_densify<double><<<gdn, 256, 0, h->stream>>>(h->A64, h->nbr, h->ne, nb, M, n);
    ++launches;
    const int np = lu_factor<double>(h, M, perms, nn, pdl, &launches);
    double* Di = reinterpret_cast<double*>(dinv);
    dg_launch(h, pdl, k_lu_diag_inv<double>, dim3(nbk), dim3(32), (const double*)M, nn, Di);
    dg_launch_smem(h, pdl, sizeof(double) * n, k_lu_solve<double>, dim3(1), dim3(LU_SOLVE_THREADS), (const double*)M,
                   (const double*)Di, (const int*)perms, np, (const double*)Fv, x, nn, 0, norms);
    launches += 2;
    h->nlaunch += launches;
    DG_LAUNCH_CK(h);
    int flag = 0;
    DG_CK(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flag) return dg_fail(h, DG_ERR_SINGULAR_BLOCK, "singular matrix in the dense solve");
    return DG_OK;
}
