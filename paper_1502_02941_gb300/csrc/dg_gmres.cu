// dg_gmres.cu -- device-resident restarted GMRES(m) with right preconditioning
// (Saad & Schultz 1986), replacing the paper's direct solve Stiff\F.
//
// Every step of the iteration runs in kernels on the handle's stream; the
// host only launches one captured CUDA graph per restart cycle and reads a
// small status header when the cycle ends.  One Arnoldi step j:
//   Z       = s_j M^-1 V_j                 (block-Jacobi apply, lazily scaled)
//   V_{j+1} = A Z                          (operator apply)
//   h_d     = s_d <V_d, V_{j+1}>, d <= j, and ||V_{j+1}||^2  (one fused multi-dot pass)
//   V_{j+1} -= sum_d h_d s_d V_d, ||V_{j+1}||^2               (one update pass)
//   [if the norm fell below 0.7 of its value before: a second classical
//    Gram-Schmidt pass ("twice is enough")]
//   Hessenberg column, Givens rotations, residual estimate   (one thread)
// Basis vectors are stored unnormalised with s_i = 1/||V_i|| so no separate
// normalisation pass is needed.  All Hessenberg/Givens arithmetic is f64.
// At the end of a cycle: y = H^-1 g (one thread), U = sum y_i s_i V_i,
// x += M^-1 U, r = F - A x, and the true residual decides convergence.
#include <math.h>
#include <string.h>

#include "dg_kernels.cuh"

struct GmresState {  // header fields first: the first GM_HDR bytes go to the host
    int active;      // Arnoldi steps proceed while 1
    int j;           // steps completed in the current cycle
    int its;         // total Arnoldi steps
    int cycles;      // completed restart cycles
    int converged;   // true residual <= tol
    int done;        // solver finished (converged, capped, or failed)
    int reorth;      // second Gram-Schmidt pass requested for this step
    int pending;     // the cycle has a correction to add to x
    int nonfinite;   // NaN/Inf met
    int m, max_it;
    int pad_;
    double tol, bnorm, relres, wn2_before;
    double scale[DG_MAXM + 2];
    double hcol[DG_MAXM + 2];
    double coef[DG_MAXM + 2];
    double H[(DG_MAXM + 1) * DG_MAXM];  // column-major, leading dimension DG_MAXM+1
    double cs[DG_MAXM], sn[DG_MAXM], g[DG_MAXM + 1], y[DG_MAXM];
};

#define GM_G 4   // dots per block in the multi-dot kernel
#define GM_HDR 96  // bytes of GmresState copied back to the host (through relres)

// ---------------------------------------------------------------------------
// reduction helper: 4 block sums at once (blockDim.x == 256)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum4(double* v, double (*sh)[8]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < GM_G; ++g) v[g] = dg_warp_sum(v[g]);
    if (lane == 0)
#pragma unroll
        for (int g = 0; g < GM_G; ++g) sh[g][wid] = v[g];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int g = 0; g < GM_G; ++g) {
            double t = lane < 8 ? sh[g][lane] : 0.0;
            v[g] = dg_warp_sum(t);
        }
    }
}

// x = 0, V_0 = F, partial ||F||^2
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_init(const TV* __restrict__ F, TV* __restrict__ x, TV* __restrict__ V0,
                                                  long n, double* partials) {
    __shared__ double sh[GM_G][8];
    double v[GM_G] = {0, 0, 0, 0};
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const TV f = F[l];
        x[l] = (TV)0;
        V0[l] = f;
        v[0] += (double)f * (double)f;
    }
    block_sum4(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

__device__ double reduce_partials(const double* p, int cnt, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s += p[i];
    return dg_block_sum(s, sh);
}

__global__ void k_gm_ctl_init(GmresState* st, const double* partials, int gx, int m, int max_it, double tol) {
    __shared__ double sh[32];
    const double b2 = reduce_partials(partials, gx, sh);
    if (threadIdx.x != 0) return;
    st->m = m;
    st->max_it = max_it;
    st->tol = tol;
    st->its = 0;
    st->cycles = 0;
    st->reorth = 0;
    st->pending = 0;
    st->nonfinite = 0;
    st->j = 0;
    const double bn = sqrt(b2);
    st->bnorm = bn;
    if (!isfinite(bn)) {
        st->nonfinite = 1;
        st->done = 1;
        st->active = 0;
        st->converged = 0;
        st->relres = bn;
        return;
    }
    if (bn == 0.0) {
        st->done = 1;
        st->converged = 1;
        st->active = 0;
        st->relres = 0.0;
        return;
    }
    st->relres = 1.0;
    st->converged = 0;
    st->done = tol >= 1.0 ? 1 : 0;
    st->converged = st->done;
    st->active = st->done ? 0 : 1;
    for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
    st->g[0] = bn;
    st->scale[0] = 1.0 / bn;
}

// Multi-dot: raw r_d = <V_d, V_{j+1}> for d <= j (pass 1 also d = j+1: the norm).
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_dots(const TV* __restrict__ V, long n, const GmresState* st,
                                                  double* partials, int gx, int pass) {
    if (!st->active || (pass == 2 && !st->reorth)) return;
    const int j = st->j;
    const int dlast = pass == 1 ? j + 1 : j;
    const int d0 = blockIdx.y * GM_G;
    if (d0 > dlast) return;
    __shared__ double sh[GM_G][8];
    const TV* __restrict__ w = V + (long)(j + 1) * n;
    const TV* vp[GM_G];
#pragma unroll
    for (int g = 0; g < GM_G; ++g) vp[g] = V + (long)min(d0 + g, j + 1) * n;
    double v[GM_G] = {0, 0, 0, 0};
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gx * blockDim.x) {
        const double wl = (double)w[l];
#pragma unroll
        for (int g = 0; g < GM_G; ++g)
            if (d0 + g <= dlast) v[g] += (double)vp[g][l] * wl;
    }
    block_sum4(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int g = 0; g < GM_G; ++g)
            if (d0 + g <= dlast) partials[(long)(d0 + g) * gx + blockIdx.x] = v[g];
}

// One warp per dot: warp w sums partials of d = w, w+32, ... (blockDim 1024).
__global__ void k_gm_ctl_dots(GmresState* st, const double* partials, int gx, int pass) {
    if (!st->active || (pass == 2 && !st->reorth)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = st->j;
    const int dlast = pass == 1 ? j + 1 : j;
    for (int d = wid; d <= dlast; d += nw) {
        double r = 0.0;
        for (int i = lane; i < gx; i += 32) r += partials[(long)d * gx + i];
        r = dg_warp_sum(r);
        if (lane == 0) {
            if (d == j + 1) {
                st->wn2_before = r;
            } else {
                const double hd = st->scale[d] * r;
                st->hcol[d] = pass == 1 ? hd : st->hcol[d] + hd;
                st->coef[d] = hd * st->scale[d];
            }
        }
    }
}

// V_{j+1} -= sum_{d<=j} coef_d V_d ; partial ||V_{j+1}||^2
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_update(TV* V, long n, const GmresState* st,
                                                    double* partials, int pass) {
    if (!st->active || (pass == 2 && !st->reorth)) return;
    __shared__ double c[DG_MAXM + 2];
    __shared__ double sh[GM_G][8];
    const int j = st->j;
    for (int d = threadIdx.x; d <= j; d += blockDim.x) c[d] = st->coef[d];
    __syncthreads();
    TV* w = V + (long)(j + 1) * n;   // aliases V: no __restrict__
    double v[GM_G] = {0, 0, 0, 0};
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        double acc = (double)w[l];
        int d = 0;
        for (; d + 4 <= j + 1; d += 4) {
            const double a0 = (double)V[(long)d * n + l], a1 = (double)V[(long)(d + 1) * n + l];
            const double a2 = (double)V[(long)(d + 2) * n + l], a3 = (double)V[(long)(d + 3) * n + l];
            acc -= c[d] * a0 + c[d + 1] * a1 + c[d + 2] * a2 + c[d + 3] * a3;
        }
        for (; d <= j; ++d) acc -= c[d] * (double)V[(long)d * n + l];
        const TV out = (TV)acc;
        w[l] = out;
        v[0] += (double)out * (double)out;
    }
    block_sum4(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// Norm, re-orthogonalisation decision, Hessenberg column, Givens rotation.
__global__ void k_gm_ctl_update(GmresState* st, const double* partials, int gx, int pass) {
    if (!st->active || (pass == 2 && !st->reorth)) return;
    __shared__ double sh[32];
    const double wn2 = reduce_partials(partials, gx, sh);
    if (threadIdx.x != 0) return;
    const int j = st->j;
    const double wn = sqrt(wn2);
    if (pass == 1 && wn < 0.7 * sqrt(st->wn2_before)) {
        st->reorth = 1;
        return;
    }
    st->reorth = 0;
    const int LD = DG_MAXM + 1;
    double* Hc = st->H + (long)j * LD;
    for (int i = 0; i <= j; ++i) Hc[i] = st->hcol[i];
    Hc[j + 1] = wn;
    for (int i = 0; i < j; ++i) {
        const double t1 = st->cs[i] * Hc[i] + st->sn[i] * Hc[i + 1];
        const double t2 = -st->sn[i] * Hc[i] + st->cs[i] * Hc[i + 1];
        Hc[i] = t1;
        Hc[i + 1] = t2;
    }
    const double a = Hc[j], b = Hc[j + 1];
    const double r = hypot(a, b);
    const double c = r == 0.0 ? 1.0 : a / r, s = r == 0.0 ? 0.0 : b / r;
    st->cs[j] = c;
    st->sn[j] = s;
    Hc[j] = r;
    Hc[j + 1] = 0.0;
    st->g[j + 1] = -s * st->g[j];
    st->g[j] = c * st->g[j];
    st->scale[j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
    st->its += 1;
    st->j = j + 1;
    st->pending = 1;
    const bool bad = !isfinite(wn) || !isfinite(r);
    if (bad) st->nonfinite = 1;
    const double est = fabs(st->g[j + 1]);
    const bool breakdown = !(wn > 1e-300) || !(r > 0.0);
    if (bad || est <= st->tol * st->bnorm || j + 1 >= st->m || st->its >= st->max_it || breakdown) st->active = 0;
}

// y = H(0:jj,0:jj)^-1 g(0:jj); coef_i = y_i s_i
__global__ void k_gm_ctl_solve(GmresState* st) {
    if (threadIdx.x != 0 || !st->pending) return;
    const int jj = st->j;
    const int LD = DG_MAXM + 1;
    for (int i = jj - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int l = i + 1; l < jj; ++l) s -= st->H[(long)l * LD + i] * st->y[l];
        const double d = st->H[(long)i * LD + i];
        st->y[i] = d != 0.0 ? s / d : 0.0;
    }
    for (int i = 0; i < jj; ++i) st->coef[i] = st->y[i] * st->scale[i];
}

// U = sum_{i<jj} coef_i V_i
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_combine(const TV* __restrict__ V, long n, const GmresState* st,
                                                     TV* __restrict__ U) {
    if (!st->pending) return;
    __shared__ double c[DG_MAXM + 2];
    const int jj = st->j;
    for (int d = threadIdx.x; d < jj; d += blockDim.x) c[d] = st->coef[d];
    __syncthreads();
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int d = 0; d < jj; ++d) acc += c[d] * (double)V[(long)d * n + l];
        U[l] = (TV)acc;
    }
}

template <typename TV>
__global__ void __launch_bounds__(256) k_gm_axpy(TV* __restrict__ x, const TV* __restrict__ z, long n,
                                                  const GmresState* st) {
    if (!st->pending) return;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        x[l] = (TV)((double)x[l] + (double)z[l]);
}

// V_0 = F - AX ; partial norm
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_resid(const TV* __restrict__ F, const TV* __restrict__ AX,
                                                   TV* __restrict__ V0, long n, const GmresState* st,
                                                   double* partials) {
    if (!st->pending) return;
    __shared__ double sh[GM_G][8];
    double v[GM_G] = {0, 0, 0, 0};
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const double r = (double)F[l] - (double)AX[l];
        const TV rv = (TV)r;
        V0[l] = rv;
        v[0] += (double)rv * (double)rv;
    }
    block_sum4(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

__global__ void k_gm_ctl_restart(GmresState* st, const double* partials, int gx) {
    if (!st->pending) return;
    __shared__ double sh[32];
    const double r2 = reduce_partials(partials, gx, sh);
    if (threadIdx.x != 0) return;
    const double beta = sqrt(r2);
    st->pending = 0;
    st->cycles += 1;
    st->relres = beta / st->bnorm;
    st->j = 0;
    if (!isfinite(beta) || st->nonfinite) {
        st->nonfinite = 1;
        st->done = 1;
        st->active = 0;
        return;
    }
    if (st->relres <= st->tol) {
        st->converged = 1;
        st->done = 1;
        st->active = 0;
        return;
    }
    if (st->its >= st->max_it) {
        st->done = 1;
        st->active = 0;
        return;
    }
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = beta;
    st->scale[0] = 1.0 / beta;
    st->active = 1;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int NB, typename TA, typename TV>
static void launch_apply(dg_handle* h, const TA* A, const TV* x, TV* y, DevCtl ctl, VecSel sx, VecSel sy) {
    const unsigned grid = (unsigned)((h->ne + 255) / 256);
    k_apply<NB, TA, TV, TV><<<grid, 256, 0, h->stream>>>(A, h->nbr, x, y, h->ne, ctl, sx, sy);
}
template <int NB, typename TB, typename TV>
static void launch_bj(dg_handle* h, const TB* B, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz) {
    const unsigned grid = (unsigned)((h->ne + 255) / 256);
    k_bj_apply<NB, TB, TV, TV><<<grid, 256, 0, h->stream>>>(B, r, z, h->ne, ctl, sr, sz);
}

struct GmSetup {
    long n;
    int m;
    int gx;
};

// One restart cycle: m Arnoldi steps, the correction and the true residual.
template <int NB, typename TA, typename TB, typename TV>
static int enqueue_cycle(dg_handle* h, const GmSetup& S, const TA* A, const TB* B, const TV* F, TV* x) {
    TV* V = (TV*)h->V;
    TV* Z = (TV*)h->Z;
    TV* R = (TV*)h->R;
    GmresState* st = h->st;
    const long n = S.n;
    const int gx = S.gx;
    const int gy = (S.m + 2 + GM_G - 1) / GM_G;
    const dim3 gdots(gx, gy);
    DevCtl step{&st->active, st->scale};
    DevCtl step_noscale{&st->active, nullptr};
    VecSel vj{&st->j, 0, n}, vj1{&st->j, 1, n};
    for (int it = 0; it < S.m; ++it) {
        launch_bj<NB, TB, TV>(h, B, V, Z, step, vj, vsel_fixed());
        launch_apply<NB, TA, TV>(h, A, Z, V, step_noscale, vsel_fixed(), vj1);
        for (int pass = 1; pass <= 2; ++pass) {
            k_gm_dots<TV><<<gdots, 256, 0, h->stream>>>(V, n, st, h->partials, gx, pass);
            k_gm_ctl_dots<<<1, 1024, 0, h->stream>>>(st, h->partials, gx, pass);
            k_gm_update<TV><<<gx, 256, 0, h->stream>>>(V, n, st, h->partials, pass);
            k_gm_ctl_update<<<1, 256, 0, h->stream>>>(st, h->partials, gx, pass);
        }
    }
    DevCtl pend{&st->pending, nullptr};
    k_gm_ctl_solve<<<1, 32, 0, h->stream>>>(st);
    k_gm_combine<TV><<<gx, 256, 0, h->stream>>>(V, n, st, R);
    launch_bj<NB, TB, TV>(h, B, R, Z, pend, vsel_fixed(), vsel_fixed());
    k_gm_axpy<TV><<<gx, 256, 0, h->stream>>>(x, Z, n, st);
    launch_apply<NB, TA, TV>(h, A, x, R, pend, vsel_fixed(), vsel_fixed());
    k_gm_resid<TV><<<gx, 256, 0, h->stream>>>(F, R, V, n, st, h->partials);
    k_gm_ctl_restart<<<1, 256, 0, h->stream>>>(st, h->partials, gx);
    // status header to pinned host memory
    cudaMemcpyAsync(h->st_host, st, GM_HDR, cudaMemcpyDeviceToHost, h->stream);
    return 10 * S.m + 7;   // kernels enqueued
}

static dg_status ensure_workspace(dg_handle* h, long n, int m, size_t elem) {
    const size_t need_v = (size_t)(m + 2) * n * elem;
    dg_status s;
    if (h->gm_n != (size_t)n || h->gm_m != m || !h->V) {
        if ((s = dg_realloc(h, (void**)&h->V, need_v)) != DG_OK) return s;
        if ((s = dg_realloc(h, (void**)&h->Z, (size_t)n * 8)) != DG_OK) return s;
        if ((s = dg_realloc(h, (void**)&h->R, (size_t)n * 8)) != DG_OK) return s;
        h->gm_n = n;
        h->gm_m = m;
        if (h->gm_graph) {
            cudaGraphExecDestroy(h->gm_graph);
            h->gm_graph = nullptr;
        }
    }
    if (!h->partials)
        if ((s = dg_realloc(h, (void**)&h->partials, sizeof(double) * (DG_MAXM + 2) * 4096)) != DG_OK) return s;
    if (!h->st)
        if ((s = dg_realloc(h, (void**)&h->st, sizeof(GmresState))) != DG_OK) return s;
    if (!h->st_host) DG_CK(h, cudaMallocHost((void**)&h->st_host, sizeof(GmresState)));
    return DG_OK;
}

static int grid_x(dg_handle* h, long n) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    long want = (long)sms * 4;
    long cap = (n + 255) / 256;
    long g = want < cap ? want : cap;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (int)g;
}

template <int NB, typename TA, typename TB, typename TV>
static dg_status gmres_run(dg_handle* h, const TA* A, const TB* B, const TV* F, TV* x, dg_solve_info* info) {
    const long n = (long)h->ne * NB;
    const int m = h->p.gmres_m;
    dg_status s = ensure_workspace(h, n, m, sizeof(TV));
    if (s != DG_OK) return s;
    GmSetup S{n, m, grid_x(h, n)};
    // initialise
    k_gm_init<TV><<<S.gx, 256, 0, h->stream>>>(F, x, (TV*)h->V, n, h->partials);
    k_gm_ctl_init<<<1, 256, 0, h->stream>>>(h->st, h->partials, S.gx, m, h->p.max_it, h->p.tol);
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(h->st_host, h->st, GM_HDR, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    // capture one cycle into a graph keyed on the buffers it touches
    const int key[4] = {(int)(((uintptr_t)x) & 0x7fffffff), (int)(((uintptr_t)F) & 0x7fffffff),
                        (int)(((uintptr_t)A) & 0x7fffffff), (int)(((uintptr_t)B) & 0x7fffffff) ^ m};
    if (h->gm_graph && memcmp(key, h->gm_graph_key, sizeof(key)) != 0) {
        cudaGraphExecDestroy(h->gm_graph);
        h->gm_graph = nullptr;
    }
    const bool use_graph = h->stream != nullptr;  // capture needs a non-legacy stream
    if (use_graph && !h->gm_graph) {
        cudaGraph_t g;
        DG_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->gm_nodes = enqueue_cycle<NB, TA, TB, TV>(h, S, A, B, F, x);
        DG_CK(h, cudaStreamEndCapture(h->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&h->gm_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return dg_cuda_fail(h, e, "cudaGraphInstantiate");
        memcpy(h->gm_graph_key, key, sizeof(key));
    }
    const int max_cycles = h->p.max_it + 2;
    for (int c = 0; c < max_cycles && !h->st_host->done; ++c) {
        if (use_graph) {
            DG_CK(h, cudaGraphLaunch(h->gm_graph, h->stream));
            h->nlaunch += h->gm_nodes;
        } else {
            h->nlaunch += enqueue_cycle<NB, TA, TB, TV>(h, S, A, B, F, x);
        }
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaStreamSynchronize(h->stream));
    }
    GmresState* hs = h->st_host;
    if (info) {
        info->iterations = hs->its;
        info->restarts = hs->cycles;
        info->outer = 0;
        info->relres = hs->relres;
        info->status = hs->converged ? DG_OK : DG_NOT_CONVERGED;
    }
    if (hs->nonfinite) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the GMRES iteration");
    if (!hs->converged) return dg_fail(h, DG_NOT_CONVERGED, "GMRES reached the iteration cap");
    return DG_OK;
}

template <int NB>
static dg_status gmres_f64(dg_handle* h, const double* F, double* x, dg_solve_info* info) {
    const double* B = h->p.precond == DG_PRECOND_BLOCK_JACOBI ? h->Binv64 : nullptr;
    return gmres_run<NB, double, double, double>(h, h->A64, B, F, x, info);
}

extern "C" dg_status dg_gmres_solve(dg_handle* h, const double* F, double* x, dg_solve_info* info) {
    if (!h || !x) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "f64 blocks not stored");
    if (h->p.precond == DG_PRECOND_BLOCK_JACOBI && !h->bj_ok) {
        dg_status s = dg_precond_setup(h, DG_PRECOND_BLOCK_JACOBI);
        if (s != DG_OK) return s;
    }
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    if (!dg_aligned16(F) || !dg_aligned16(x)) return dg_fail(h, DG_ERR_INVALID_ARG, "F and x must be 16-byte aligned");
    switch (dg_nb(h->asm_k)) {
        case 3: return gmres_f64<3>(h, F, x, info);
        case 6: return gmres_f64<6>(h, F, x, info);
        case 10: return gmres_f64<10>(h, F, x, info);
    }
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}
