// dg_gmres.cu -- device-resident restarted GMRES(m) with right preconditioning
// (Saad & Schultz 1986), replacing the paper's direct solve Stiff\F.
//
// Every step of the iteration runs in kernels on the handle's stream; the
// host launches one captured CUDA graph per restart cycle and reads a small
// status header when the cycle ends.  One Arnoldi step j is 3 kernels:
//   1. V_{j+1} = s_j (A M^-1) V_j                   (one apply of the operator
//                                                    preconditioned once at
//                                                    set-up; with Schwarz or
//                                                    the learned correction the
//                                                    preconditioner is applied
//                                                    first, then A)
//   2. r_d = <V_d, V_{j+1}>, d <= j+1               (one multi-dot pass; d = j+1
//                                                    is ||w||^2)
//   3. V_{j+1} -= sum_d s_d^2 r_d V_d               (one update pass)
// The norm of the orthogonalised vector comes from the same reduction as
// ||w||^2 - sum_d h_d^2 (single-reduction classical Gram-Schmidt).  When that
// leaves less than DG_REORTH_FRAC ||w||^2 a second Gram-Schmidt pass runs (kernels 2-3
// again, which otherwise exit at once) and its own self-dot gives the norm.
// The multi-dot finishes its reduction in the last block to arrive
// (threadfence + arrival counter, no waiting), which sums the per-block
// partials in a fixed order, so results are deterministic; block 0 of the
// update kernel then takes the Hessenberg / Givens step and the convergence
// decision while the other blocks stream.  Basis vectors are stored
// unnormalised with s_i = 1/||V_i||.  Hessenberg and Givens arithmetic is f64.
// End of a cycle: y = H^-1 g, U = sum y_i s_i V_i, x += M^-1 U, r = F - A x,
// and the true residual decides convergence.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "dg_kernels.cuh"

template <typename TV>
dg_status dg_mlp_correct(dg_handle* h, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz, const int* iuse);

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
    unsigned int arrive;  // last-block arrival counter
    int jw;          // column being orthogonalised (read by the update kernel)
    int colready;    // the column's norm is known; the update kernel takes the Givens step
    double wn_fin;   // that norm
    double tol, bnorm, relres;
    double scale[DG_MAXM + 2];
    double hcol[DG_MAXM + 2];
    double coef[DG_MAXM + 2];
    double H[(DG_MAXM + 1) * DG_MAXM];  // column-major, leading dimension DG_MAXM+1
    double cs[DG_MAXM], sn[DG_MAXM], g[DG_MAXM + 1], y[DG_MAXM];
};

#define GM_HDR 96     // bytes of GmresState copied back to the host (through relres)
#define GM_TX 32      // multi-dot block: 32 vector entries x 32 dot groups
#define GM_TY 32
#define GM_DPT ((DG_MAXM + 2 + GM_TY - 1) / GM_TY)   // dots per thread

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Per-thread accumulation: f64 vectors accumulate in f64; f32 vectors in f32
// with Kahan compensation (the block/grid reduction is always f64).
template <typename TV>
struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void fma(double a, double b) { s = ::fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void fma(float a, float b) {
        const float y = a * b - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// 16-byte vector of basis entries.  Basis vectors have a padded leading
// dimension (a multiple of 64 entries) and zero padding, so every vector is
// 16-byte aligned and the kernels below may run over whole 16-byte vectors.
template <typename TV>
struct Vec;
template <>
struct Vec<double> {
    using T = double2;
    static constexpr int W = 2;
    __device__ __forceinline__ static double get(const T& v, int i) { return i == 0 ? v.x : v.y; }
    __device__ __forceinline__ static void set(T& v, int i, double a) { if (i == 0) v.x = a; else v.y = a; }
};
template <>
struct Vec<float> {
    using T = float4;
    static constexpr int W = 4;
    __device__ __forceinline__ static float get(const T& v, int i) {
        return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    }
    __device__ __forceinline__ static void set(T& v, int i, float a) {
        if (i == 0) v.x = a; else if (i == 1) v.y = a; else if (i == 2) v.z = a; else v.w = a;
    }
};

// Returns true in exactly one block: the last to arrive.  All partial results
// written before the call by any block are visible to that block (read them
// with __ldcg).  The counter is reset for the next kernel.
__device__ __forceinline__ bool last_block(unsigned int* counter) {
    __shared__ int amlast;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int nblk = gridDim.x * gridDim.y;
        const unsigned int t = atomicAdd(counter, 1u);
        amlast = (t == nblk - 1) ? 1 : 0;
        if (amlast) *counter = 0u;
    }
    __syncthreads();
    return amlast != 0;
}

// Sum cnt partials with all threads of a 1-D block; every thread gets it.
__device__ double sum_partials(const double* p, int cnt, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s += __ldcg(p + i);
    return dg_block_sum(s, sh);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// x = 0, V_0 = F; last block: ||F||, state initialisation.
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_init(const TV* __restrict__ F, TV* __restrict__ x, TV* __restrict__ V0,
                                                  long n, GmresState* st, double* partials, int m, int max_it,
                                                  double tol) {
    __shared__ double sh[32];
    Acc<TV> a;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const TV f = F[l];
        x[l] = (TV)0;
        V0[l] = f;
        a.fma(f, f);
    }
    const double v = dg_block_sum(a.get(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
    if (!last_block(&st->arrive)) return;
    const double b2 = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x != 0) return;
    st->m = m;
    st->max_it = max_it;
    st->tol = tol;
    st->its = 0;
    st->cycles = 0;
    st->reorth = 0;
    st->colready = 0;
    st->pending = 0;
    st->nonfinite = 0;
    st->j = 0;
    const double bn = sqrt(b2);
    st->bnorm = bn;
    st->converged = 0;
    if (!isfinite(bn)) {
        st->nonfinite = 1;
        st->done = 1;
        st->active = 0;
        st->relres = bn;
        return;
    }
    if (bn == 0.0 || tol >= 1.0) {
        st->done = 1;
        st->converged = 1;
        st->active = 0;
        st->relres = 0.0;
        return;
    }
    st->relres = 1.0;
    st->done = 0;
    st->active = 1;
    for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
    st->g[0] = bn;
    st->scale[0] = 1.0 / bn;
}
// Givens / Hessenberg step for column j; runs in thread 0 of the update
// kernel's block 0 with the column and the previous rotations staged in
// shared memory.
__device__ void gm_finish_column(GmresState* st, double wn, const double* hc, const double* cs, const double* sn) {
    // state read up front: the stores into H below may alias it for the compiler
    const int j = st->j, m = st->m, its = st->its + 1, max_it = st->max_it;
    const double gj = st->g[j], tolb = st->tol * st->bnorm;
    const int LD = DG_MAXM + 1;
    double* Hc = st->H + (long)j * LD;
    double a = hc[0];
    for (int i = 0; i < j; ++i) {
        const double b = hc[i + 1];
        Hc[i] = cs[i] * a + sn[i] * b;
        a = -sn[i] * a + cs[i] * b;
    }
    const double r = hypot(a, wn);
    const double ir = r == 0.0 ? 0.0 : 1.0 / r;
    const double c = r == 0.0 ? 1.0 : a * ir, s = wn * ir;
    st->cs[j] = c;
    st->sn[j] = s;
    Hc[j] = r;
    Hc[j + 1] = 0.0;
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->scale[j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
    st->its = its;
    st->j = j + 1;
    st->pending = 1;
    const bool bad = !isfinite(wn) || !isfinite(r);
    if (bad) st->nonfinite = 1;
    const double est = fabs(s * gj);
    const bool breakdown = !(wn > 1e-300) || !(r > 0.0);
    if (bad || est <= tolb || j + 1 >= m || its >= max_it || breakdown) st->active = 0;
}


// Multi-dot r_d = <V_d, V_{j+1}>, d <= dlast (pass 1: dlast = j+1, the last
// one being the squared norm; pass 2: dlast = j).  One 1024-thread block per
// SM, block (32, 32): lanes run over 32 consecutive entries, warp ty over the
// dots d = ty, ty + 32, ...; four chunks per loop trip keep ~10 loads in
// flight per thread.  Last block: all threads reduce the per-block partials
// (16 threads per dot, independent loads), then h_d = s_d r_d into hcol and the
// update coefficients s_d h_d.
template <typename TV>
__global__ void __launch_bounds__(GM_TX* GM_TY) k_gm_dots(const TV* __restrict__ V, long ld, long nvec,
                                                         GmresState* st, double* partials, int pass) {
    if constexpr (sizeof(TV) == 4) {   // programmatic dependent launch (f32 solves)
        dg_grid_release();
        dg_grid_wait();
    }
    if (!st->active || (pass == 2 && !st->reorth)) return;
    using VT = typename Vec<TV>::T;
    constexpr int W = Vec<TV>::W;
    const int j = st->j;
    const int dlast = j + 1;            // V_0..V_j and w itself
    const int tx = threadIdx.x, ty = threadIdx.y;
    const VT* __restrict__ w = reinterpret_cast<const VT*>(V + (long)(j + 1) * ld);
    Acc<TV> acc[GM_DPT];
    const long nchunk = (nvec + GM_TX - 1) / GM_TX;
    // with at most 16 dots, nsub = 32 / ncol warps share each dot (interleaved
    // chunks), so every warp streams whatever the step j
    const int ncol = dlast + 1;
    const int nsub = ncol <= GM_TY / 2 ? GM_TY / ncol : 1;
    const int dsel = nsub > 1 ? ty % ncol : ty;
    const int sub = nsub > 1 ? ty / ncol : 0;
    const bool live = ty < ncol * nsub || nsub == 1;
    const long step = (long)gridDim.x * nsub;
    for (long c = blockIdx.x + (long)sub * gridDim.x; live && c < nchunk; c += 4 * step) {
        VT wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long q = (c + u * step) * GM_TX + tx;
            if (q < nvec) wv[u] = w[q];
            else
#pragma unroll
                for (int i = 0; i < W; ++i) Vec<TV>::set(wv[u], i, (TV)0);
        }
#pragma unroll
        for (int k = 0; k < GM_DPT; ++k) {
            const int d = dsel + GM_TY * k;
            if (d <= dlast) {
                const VT* __restrict__ vd = reinterpret_cast<const VT*>(V + (long)d * ld);
                VT v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long q = (c + u * step) * GM_TX + tx;
                    if (q < nvec) v[u] = vd[q];
                    else
#pragma unroll
                        for (int i = 0; i < W; ++i) Vec<TV>::set(v[u], i, (TV)0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[k].fma(Vec<TV>::get(v[u], i), Vec<TV>::get(wv[u], i));
            }
        }
    }
    const int gx = gridDim.x;
    if (nsub > 1) {
        __shared__ double ws[GM_TY];
        const double v = dg_warp_sum(acc[0].get());
        if (tx == 0) ws[ty] = live ? v : 0.0;
        __syncthreads();
        const int t0 = ty * GM_TX + tx;
        if (t0 < ncol) {
            double r = 0.0;
            for (int u = 0; u < nsub; ++u) r += ws[t0 + u * ncol];
            partials[(long)t0 * gx + blockIdx.x] = r;
        }
    } else {
        // only the accumulators that hold a dot are reduced (warp-uniform test):
        // every f64 instruction here costs time on this GPU's FP64 pipe
#pragma unroll
        for (int k = 0; k < GM_DPT; ++k) {
            const int d = ty + GM_TY * k;
            if (d <= dlast) {
                const double v = dg_warp_sum(acc[k].get());
                if (tx == 0) partials[(long)d * gx + blockIdx.x] = v;
            }
        }
    }
    if (!last_block(&st->arrive)) return;
    // 16 threads per dot: thread t sums partials t%16, t%16+16, ... of dot t/16
    __shared__ double hp[DG_MAXM + 2];
    const int t = ty * GM_TX + tx;
    for (int d0 = 0; d0 <= dlast; d0 += (GM_TX * GM_TY) / 16) {
        const int d = d0 + t / 16;
        double r = 0.0;
        if (d <= dlast) {
#pragma unroll 4
            for (int b = t % 16; b < gx; b += 16) r += __ldcg(partials + (long)d * gx + b);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((t % 16) == 0 && d <= dlast) {
            if (d == j + 1) {
                hp[d] = r;                    // ||w||^2
            } else {
                const double hd = st->scale[d] * r;
                hp[d] = hd;
                st->hcol[d] = pass == 1 ? hd : st->hcol[d] + hd;
                st->coef[d] = hd * st->scale[d];
            }
        }
    }
    __syncthreads();
    if (t >= 32) return;
    // norm of w - sum h_d v_d without another pass: ||w||^2 - sum h_d^2 (the
    // v_d are orthonormal).  Accepted when at least DG_REORTH_FRAC ||w||^2
    // remains (at most a factor 2 of cancellation in the norm); otherwise a
    // second Gram-Schmidt pass runs and its own self-dot gives the norm exactly.
    double s2 = 0.0;
    for (int d = t; d <= j; d += 32) s2 = fma(hp[d], hp[d], s2);
    s2 = dg_warp_sum(s2);
    if (t != 0) return;
    const double w2 = hp[j + 1];
    const double rest = w2 - s2;
    st->jw = j;
    if (pass == 1) {
        const bool again = !(rest >= DG_REORTH_FRAC * w2);
        st->reorth = again ? 1 : 0;
        if (again) return;
    }
    st->wn_fin = sqrt(rest > 0.0 ? rest : 0.0);
    st->colready = 1;
}

// Block 0 of the update kernels: the Givens step of the column the multi-dot
// tail marked ready, with the column and the previous rotations staged in
// shared memory.
__device__ void gm_control_block(GmresState* st) {
    __shared__ double hc[DG_MAXM + 2], css[DG_MAXM], sns[DG_MAXM];
    if (!st->colready) return;
    const int jc = st->jw;
    for (int i = threadIdx.x; i <= jc; i += blockDim.x) {
        hc[i] = st->hcol[i];
        if (i < jc) {
            css[i] = st->cs[i];
            sns[i] = st->sn[i];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->colready = 0;
        gm_finish_column(st, st->wn_fin, hc, css, sns);
    }
}

// V_{j+1} -= sum_{d<=j} coef_d V_d for the column j = jw the multi-dot kernel
// prepared.  Block 0 (dispatched first) takes the Givens step of the column
// when the multi-dot tail marked it ready, in parallel with the update (the
// update does not need it; the next step does).
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_update(TV* V, long ld, long nvec, GmresState* st, int pass) {
    if constexpr (sizeof(TV) == 4) {   // programmatic dependent launch (f32 solves)
        dg_grid_release();
        dg_grid_wait();
    }
    if (blockIdx.x == 0) {
        gm_control_block(st);
        return;
    }
    if (!st->active || (pass == 2 && !st->reorth)) return;
    using VT = typename Vec<TV>::T;
    constexpr int W = Vec<TV>::W;
    __shared__ TV c[DG_MAXM + 2];
    const int j = st->jw;
    for (int d = threadIdx.x; d <= j; d += blockDim.x) c[d] = (TV)st->coef[d];
    __syncthreads();
    VT* w = reinterpret_cast<VT*>(V + (long)(j + 1) * ld);   // aliases V: no __restrict__
    const long nthr = (long)(gridDim.x - 1) * blockDim.x;   // block 0 is the control block
    for (long q = (long)(blockIdx.x - 1) * blockDim.x + threadIdx.x; q < nvec; q += nthr) {
        VT acc = w[q];
        int d = 0;
        for (; d + 4 <= j + 1; d += 4) {
            VT v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = reinterpret_cast<const VT*>(V + (long)(d + u) * ld)[q];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < W; ++i)
                    Vec<TV>::set(acc, i, ::fma(-c[d + u], Vec<TV>::get(v[u], i), Vec<TV>::get(acc, i)));
        }
        for (; d <= j; ++d) {
            const VT v = reinterpret_cast<const VT*>(V + (long)d * ld)[q];
#pragma unroll
            for (int i = 0; i < W; ++i) Vec<TV>::set(acc, i, ::fma(-c[d], Vec<TV>::get(v, i), Vec<TV>::get(acc, i)));
        }
        w[q] = acc;
    }
}

// ---------------------------------------------------------------------------
// f32 Arnoldi kernels (the inner GMRES of the mixed-precision solvers)
// ---------------------------------------------------------------------------
#define GM32_THREADS 512
#define GM32_WARPS (GM32_THREADS / 32)
#define GM32_G 16   // dots per warp group

// f32 multi-dot r_d = <V_d, V_{j+1}>, d <= j+1 (pass 1 and pass 2 alike; d = j+1
// is ||w||^2).  The ncol = j+2 dots are cut into ngroups groups of equal size
// (at most GM32_G); the warps of a block are split into (group, row
// partition) pairs and every partition strides over the 512-byte row chunks,
// so all resident warps stream at every step j: per chunk a warp loads w once
// and the chunk of each vector of its group.  (Fewer blocks that each take an
// equal run of chunks measured slower: the kernel is latency-bound, and
// resident warps matter more than balance.)  Each lane sums its few products
// in f32, the warp in an f32 tree (32 terms); the warps of a block and then
// the blocks are summed in two-float arithmetic (f2_add), and the last block
// to arrive turns each total into one f64 value: no per-warp f64 work, which
// on this GPU's FP64 pipe would cost as much as the streaming.  The tail then
// follows the f64 kernel: h_d = s_d r_d, the update coefficients, and the norm
// ||w||^2 - sum h_d^2 or a request for a second pass.
__global__ void __launch_bounds__(GM32_THREADS, 2) k_gm_dots32(const float* __restrict__ V, long ld, long nvec,
                                                               GmresState* st, float2* partials, int pass) {
    dg_grid_release();   // programmatic dependent launch
    dg_grid_wait();
    if (!st->active || (pass == 2 && !st->reorth)) return;
    const int j = st->j;
    const int ncol = j + 2;
    const int ngroups = (ncol + GM32_G - 1) / GM32_G;   // <= 5 (ncol <= DG_MAXM + 2)
    const int gsize = (ncol + ngroups - 1) / ngroups;
    const int pb = GM32_WARPS / ngroups;                 // row partitions per block
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = wid % ngroups, part = wid / ngroups;
    const int d0 = g * gsize;
    const int dn = part < pb ? max(0, min(gsize, ncol - d0)) : 0;
    __shared__ float red[GM32_WARPS][GM32_G];
    float acc[GM32_G];
#pragma unroll
    for (int i = 0; i < GM32_G; ++i) acc[i] = 0.f;
    if (dn > 0) {
        const long nchunk = (nvec + 31) / 32;
        const long P = (long)gridDim.x * pb;
        const long ld4 = ld / 4;
        const float4* __restrict__ w = reinterpret_cast<const float4*>(V + (long)(j + 1) * ld);
        const float4* __restrict__ vg = reinterpret_cast<const float4*>(V + (long)d0 * ld);
        for (long c = (long)blockIdx.x * pb + part; c < nchunk; c += P) {
            const long q = c * 32 + lane;
            if (q >= nvec) continue;
            const float4 wv = w[q];
#pragma unroll
            for (int d = 0; d < GM32_G; ++d) {
                if (d < dn) {
                    const float4 v = vg[(long)d * ld4 + q];
                    acc[d] = fmaf(v.x, wv.x, acc[d]);
                    acc[d] = fmaf(v.y, wv.y, acc[d]);
                    acc[d] = fmaf(v.z, wv.z, acc[d]);
                    acc[d] = fmaf(v.w, wv.w, acc[d]);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < GM32_G; ++d) {
        if (d < gsize) {   // block-uniform
            float v = acc[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[wid][d] = d < dn ? v : 0.f;
        }
    }
    __syncthreads();
    const int gx = gridDim.x;
    for (int d = threadIdx.x; d < ncol; d += blockDim.x) {
        const int gg = d / gsize, dd = d - gg * gsize;
        float2 s = make_float2(0.f, 0.f);
        for (int p = 0; p < pb; ++p) s = f2_add(s, make_float2(red[p * ngroups + gg][dd], 0.f));
        partials[(long)d * gx + blockIdx.x] = s;
    }
    if (!last_block(&st->arrive)) return;
    __shared__ float2 tot[DG_MAXM + 2];
    for (int d = wid; d < ncol; d += GM32_WARPS) {
        float2 s = make_float2(0.f, 0.f);
        for (int b = lane; b < gx; b += 32) s = f2_add(s, __ldcg(partials + (long)d * gx + b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 t;
            t.x = __shfl_xor_sync(0xffffffffu, s.x, o);
            t.y = __shfl_xor_sync(0xffffffffu, s.y, o);
            s = f2_add(s, t);
        }
        if (lane == 0) tot[d] = s;
    }
    __syncthreads();
    __shared__ double hp[DG_MAXM + 2];
    for (int d = threadIdx.x; d < ncol; d += blockDim.x) {
        const double r = (double)tot[d].x + (double)tot[d].y;
        if (d == j + 1) {
            hp[d] = r;   // ||w||^2
        } else {
            const double hd = st->scale[d] * r;
            hp[d] = hd;
            st->hcol[d] = pass == 1 ? hd : st->hcol[d] + hd;
            st->coef[d] = hd * st->scale[d];
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    double s2 = 0.0;
    for (int d = threadIdx.x; d <= j; d += 32) s2 = fma(hp[d], hp[d], s2);
    s2 = dg_warp_sum(s2);
    if (threadIdx.x != 0) return;
    const double w2 = hp[j + 1];
    const double rest = w2 - s2;
    st->jw = j;
    if (pass == 1) {
        const bool again = !(rest >= DG_REORTH_FRAC * w2);
        st->reorth = again ? 1 : 0;
        if (again) return;
    }
    st->wn_fin = sqrt(rest > 0.0 ? rest : 0.0);
    st->colready = 1;
}

// f32 Gram-Schmidt update V_{j+1} -= sum_{d<=j} coef_d V_d (j = jw): block 0
// takes the Givens step; every other thread streams one 16-byte column slice
// through the basis, GM32_U vectors per round so that that many loads are in
// flight per thread.
#define GM32_U 8
__global__ void __launch_bounds__(256) k_gm_update32(float* V, long ld, long nvec, GmresState* st, int pass) {
    dg_grid_release();   // programmatic dependent launch
    dg_grid_wait();
    if (blockIdx.x == 0) {
        gm_control_block(st);
        return;
    }
    if (!st->active || (pass == 2 && !st->reorth)) return;
    __shared__ float c[DG_MAXM + 2];
    const int j = st->jw;
    for (int d = threadIdx.x; d <= j; d += blockDim.x) c[d] = (float)st->coef[d];
    __syncthreads();
    const long ld4 = ld / 4;
    float4* w = reinterpret_cast<float4*>(V + (long)(j + 1) * ld);   // aliases V: no __restrict__
    const float4* v0 = reinterpret_cast<const float4*>(V);
    const long nthr = (long)(gridDim.x - 1) * blockDim.x;
    for (long q = (long)(blockIdx.x - 1) * blockDim.x + threadIdx.x; q < nvec; q += nthr) {
        float4 acc = w[q];
        int d = 0;
        for (; d + GM32_U <= j + 1; d += GM32_U) {
            float4 v[GM32_U];
#pragma unroll
            for (int u = 0; u < GM32_U; ++u) v[u] = v0[(long)(d + u) * ld4 + q];
#pragma unroll
            for (int u = 0; u < GM32_U; ++u) {
                const float cc = -c[d + u];
                acc.x = fmaf(cc, v[u].x, acc.x);
                acc.y = fmaf(cc, v[u].y, acc.y);
                acc.z = fmaf(cc, v[u].z, acc.z);
                acc.w = fmaf(cc, v[u].w, acc.w);
            }
        }
        for (; d <= j; ++d) {
            const float4 v = v0[(long)d * ld4 + q];
            const float cc = -c[d];
            acc.x = fmaf(cc, v.x, acc.x);
            acc.y = fmaf(cc, v.y, acc.y);
            acc.z = fmaf(cc, v.z, acc.z);
            acc.w = fmaf(cc, v.w, acc.w);
        }
        w[q] = acc;
    }
}

// Launch the multi-dot + update pair of Gram-Schmidt pass `pass`.
template <typename TV>
static void launch_gs_pass(dg_handle* h, GmresWork& W, TV* V, long ld, long nvec, bool pdl, int pass) {
    if constexpr (sizeof(TV) == 4) {
        dg_launch(h, pdl, k_gm_dots32, dim3(W.gd32), dim3(GM32_THREADS), (const float*)V, ld, nvec, W.st,
                  (float2*)W.partials, pass);
        dg_launch(h, pdl, k_gm_update32, dim3(W.gu32 + 1), dim3(256), (float*)V, ld, nvec, W.st, pass);
    } else {
        dg_launch(h, pdl, k_gm_dots<TV>, dim3(W.gsm), dim3(GM_TX, GM_TY), (const TV*)V, ld, nvec, W.st, W.partials,
                  pass);
        dg_launch(h, pdl, k_gm_update<TV>, dim3(W.gx + 1), dim3(256), V, ld, nvec, W.st, pass);
    }
}

// y = H(0:jj,0:jj)^-1 g(0:jj) by column-oriented back substitution in shared
// memory; coef_i = y_i s_i.
__global__ void __launch_bounds__(256) k_gm_solve(GmresState* st, int flexible) {
    if (!st->pending) return;
    __shared__ double Hs[(DG_MAXM + 1) * DG_MAXM];
    __shared__ double gs[DG_MAXM + 1];
    const int jj = st->j;
    const int LD = DG_MAXM + 1;
    for (int t = threadIdx.x; t < jj * LD; t += blockDim.x) Hs[t] = st->H[t];
    for (int t = threadIdx.x; t < jj; t += blockDim.x) gs[t] = st->g[t];
    __syncthreads();
    for (int i = jj - 1; i >= 0; --i) {
        const double d = Hs[(long)i * LD + i];
        const double yi = d != 0.0 ? gs[i] / d : 0.0;
        __syncthreads();
        for (int l = threadIdx.x; l < i; l += blockDim.x) gs[l] -= Hs[(long)i * LD + l] * yi;
        if (threadIdx.x == 0) {
            st->y[i] = yi;
            // fixed preconditioner: x += M^-1 sum y_i s_i V_i;  flexible: x += sum y_i Z_i
            st->coef[i] = flexible ? yi : yi * st->scale[i];
        }
        __syncthreads();
    }
}

// U = sum_{i<jj} coef_i V_i  (U has the basis' zero padding too)
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_combine(const TV* __restrict__ V, long ld, long nvec,
                                                     const GmresState* st, TV* __restrict__ U) {
    if (!st->pending) return;
    using VT = typename Vec<TV>::T;
    constexpr int W = Vec<TV>::W;
    __shared__ TV c[DG_MAXM + 2];
    const int jj = st->j;
    for (int d = threadIdx.x; d < jj; d += blockDim.x) c[d] = (TV)st->coef[d];
    __syncthreads();
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nvec; q += (long)gridDim.x * blockDim.x) {
        VT acc;
#pragma unroll
        for (int i = 0; i < W; ++i) Vec<TV>::set(acc, i, (TV)0);
        for (int d = 0; d < jj; ++d) {
            const VT v = reinterpret_cast<const VT*>(V + (long)d * ld)[q];
#pragma unroll
            for (int i = 0; i < W; ++i) Vec<TV>::set(acc, i, ::fma(c[d], Vec<TV>::get(v, i), Vec<TV>::get(acc, i)));
        }
        reinterpret_cast<VT*>(U)[q] = acc;
    }
}

template <typename TV>
__global__ void __launch_bounds__(256) k_gm_axpy(TV* __restrict__ x, const TV* __restrict__ z, long n,
                                                  const GmresState* st) {
    if (!st->pending) return;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        x[l] = x[l] + z[l];
}

// V_0 = F - AX, ||V_0||; last block: restart decision.
template <typename TV>
__global__ void __launch_bounds__(256) k_gm_resid(const TV* __restrict__ F, const TV* __restrict__ AX,
                                                   TV* __restrict__ V0, long n, GmresState* st, double* partials) {
    if (!st->pending) return;
    __shared__ double sh[32];
    Acc<TV> a;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const TV rv = F[l] - AX[l];
        V0[l] = rv;
        a.fma(rv, rv);
    }
    const double v = dg_block_sum(a.get(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
    if (!last_block(&st->arrive)) return;
    const double r2 = sum_partials(partials, gridDim.x, sh);
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
template <int NB, typename TA, typename TV, bool UNIT = false>
static void launch_apply(dg_handle* h, const TA* A, const TV* x, TV* y, DevCtl ctl, VecSel sx, VecSel sy,
                         bool pdl = false) {
    const ElemShape es = elem_shape(h);
    dg_launch(h, pdl, k_apply<NB, TA, TV, TV, UNIT>, dim3(es.grid), dim3(es.block), A, (const int*)h->nbr, x, y,
              h->ne, ctl, sx, sy);
}
template <int NB, typename TB, typename TV>
static void launch_bj(dg_handle* h, const TB* B, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz,
                      bool pdl = false) {
    const unsigned grid = (unsigned)((h->ne + 255) / 256);
    dg_launch(h, pdl, k_bj_apply<NB, TB, TV, TV>, dim3(grid), dim3(256), B, r, z, h->ne, ctl, sr, sz);
}

// One restart cycle: m Arnoldi steps, the correction and the true residual.
// Returns the number of kernels enqueued.
template <int NB, typename TA, typename TB, typename TV>
static int enqueue_cycle(dg_handle* h, GmresWork& W, const TA* A, const TB* B, const TV* F, TV* x, bool flex,
                         const TA* Ah, const TV* G) {
    TV* V = (TV*)W.V;
    TV* Z = (TV*)W.Z;
    TV* R = (TV*)W.R;
    TV* Zb = (TV*)W.Zb;
    GmresState* st = W.st;
    const long n = (long)W.n;
    const long ld = (long)W.ld;
    const long nvec = ld / Vec<TV>::W;
    const int gx = W.gx;
    DevCtl step{&st->active, st->scale};
    DevCtl step_noscale{&st->active, nullptr};
    VecSel vj{&st->j, 0, ld}, vj1{&st->j, 1, ld};
    // f32 vectors: the Arnoldi-step kernels are launched programmatically
    // dependent on their predecessor (each waits for it before reading), so
    // launch latency and the predecessor's tail overlap.  Not for f64: the
    // early-scheduled blocks pile onto the SMs that free up first, and the
    // FP64-bound kernels then run unbalanced (measured 4.90 against 5.36
    // solves/s on the 256x256 P2 workload; f32 refinement 12.74 against 12.64)
    const bool pdl = h->pdl && h->stream != nullptr && sizeof(TV) == 4;
    int extra = 0;
    for (int it = 0; it < W.m; ++it) {
        if (flex) {
            // Z_j = s_j M_BJ^-1 V_j + MLP correction, kept for the update of x
            VecSel zj{&st->j, 0, ld};
            launch_bj<NB, TB, TV>(h, B, V, Zb, step, vj, zj, pdl);
            dg_mlp_correct<TV>(h, V, Zb, step, vj, zj, nullptr);
            launch_apply<NB, TA, TV>(h, A, Zb, V, step_noscale, zj, vj1, pdl);
            ++extra;
        } else if (G) {
            // Schwarz: Z = s_j G V_j, V_{j+1} = A Z (two applies)
            launch_apply<NB, TV, TV>(h, G, V, Z, step, vj, vsel_fixed(), pdl);
            launch_apply<NB, TA, TV>(h, A, Z, V, step_noscale, vsel_fixed(), vj1, pdl);
        } else if (Ah) {
            // V_{j+1} = s_j (A M^-1) V_j: one apply of the precomputed operator
            launch_apply<NB, TA, TV, true>(h, Ah, V, V + ld, step, vj, vj, pdl);   // unit diagonal blocks
            --extra;
        } else {
            launch_bj<NB, TB, TV>(h, B, V, Z, step, vj, vsel_fixed(), pdl);
            launch_apply<NB, TA, TV>(h, A, Z, V, step_noscale, vsel_fixed(), vj1, pdl);
        }
        for (int pass = 1; pass <= 2; ++pass) launch_gs_pass<TV>(h, W, V, ld, nvec, pdl, pass);
    }
    DevCtl pend{&st->pending, nullptr};
    k_gm_solve<<<1, 256, 0, h->stream>>>(st, flex ? 1 : 0);
    if (flex) {
        k_gm_combine<TV><<<gx, 256, 0, h->stream>>>(Zb, ld, nvec, st, R);
        k_gm_axpy<TV><<<gx, 256, 0, h->stream>>>(x, R, n, st);
    } else {
        k_gm_combine<TV><<<gx, 256, 0, h->stream>>>(V, ld, nvec, st, R);
        if (G) launch_apply<NB, TV, TV>(h, G, R, Z, pend, vsel_fixed(), vsel_fixed());
        else launch_bj<NB, TB, TV>(h, B, R, Z, pend, vsel_fixed(), vsel_fixed());
        k_gm_axpy<TV><<<gx, 256, 0, h->stream>>>(x, Z, n, st);
    }
    launch_apply<NB, TA, TV>(h, A, x, R, pend, vsel_fixed(), vsel_fixed());
    k_gm_resid<TV><<<gx, 256, 0, h->stream>>>(F, R, V, n, st, W.partials);
    cudaMemcpyAsync(W.st_host, st, GM_HDR, cudaMemcpyDeviceToHost, h->stream);
    return 6 * W.m + 6 + extra - (flex ? 1 : 0);
}

void dg_gmres_free(dg_handle* h, GmresWork* w) {
    void* ptrs[] = {w->V, w->Z, w->R, w->Zb, w->partials, w->st};
    for (void* p : ptrs) dg_dev_free(h, p);
    if (w->st_host) cudaFreeHost(w->st_host);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    *w = GmresWork();
}

static dg_status ensure_workspace(dg_handle* h, GmresWork& W, long n, int m, size_t elem) {
    dg_status s;
    if (W.n != (size_t)n || W.m != m || W.elem != elem || !W.V) {
        const size_t ld = ((size_t)n + 63) / 64 * 64;
        if ((s = dg_realloc(h, &W.V, (size_t)(m + 2) * ld * elem)) != DG_OK) return s;
        if ((s = dg_realloc(h, &W.Z, ld * elem)) != DG_OK) return s;
        if ((s = dg_realloc(h, &W.R, ld * elem)) != DG_OK) return s;
        // zero padding: no kernel writes a nonzero beyond entry n of a vector
        DG_CK(h, cudaMemsetAsync(W.V, 0, (size_t)(m + 2) * ld * elem, h->stream));
        DG_CK(h, cudaMemsetAsync(W.Z, 0, ld * elem, h->stream));
        DG_CK(h, cudaMemsetAsync(W.R, 0, ld * elem, h->stream));
        if (W.Zb) {
            dg_dev_free(h, W.Zb);
            W.Zb = nullptr;
        }
        W.ld = ld;
        W.n = n;
        W.m = m;
        W.elem = elem;
        if (W.graph) {
            cudaGraphExecDestroy(W.graph);
            W.graph = nullptr;
        }
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    long want = 4L * sms, cap = (n + 255) / 256;
    W.gx = (int)(want < cap ? want : (cap < 1 ? 1 : cap));
    W.gsm = (int)((long)sms < (n + 1023) / 1024 ? sms : ((n + 1023) / 1024 < 1 ? 1 : (n + 1023) / 1024));
    {
        // f32 kernels: 16-byte slices of 4 entries; two multi-dot blocks per SM
        // (one 512-byte chunk per warp at least), five update blocks per SM (44
        // registers a thread: all resident at once)
        const long nvec4 = (long)(((size_t)n + 63) / 64 * 64) / 4;
        const long want_d = 2L * sms, cap_d = (nvec4 + 32 * GM32_WARPS - 1) / (32 * GM32_WARPS);
        W.gd32 = (int)std::max(1L, std::min(want_d, cap_d));
        const long want_u = 5L * sms - 1, cap_u = (nvec4 + 255) / 256;   // + the control block: 5 per SM
        W.gu32 = (int)std::max(1L, std::min(want_u, cap_u));
    }
    if (!W.partials)
        if ((s = dg_realloc(h, (void**)&W.partials, sizeof(double) * (DG_MAXM + 2) * 4096)) != DG_OK) return s;
    if (!W.st) {
        if ((s = dg_realloc(h, (void**)&W.st, sizeof(GmresState))) != DG_OK) return s;
        DG_CK(h, cudaMemsetAsync(W.st, 0, sizeof(GmresState), h->stream));
    }
    if (!W.st_host) DG_CK(h, cudaMallocHost((void**)&W.st_host, sizeof(GmresState)));
    return DG_OK;
}

// The precomputed A M^-1 of the block copy of type T (NULL if not stored).
template <typename T>
static const T* ahat_of(const dg_handle* h) {
    if constexpr (sizeof(T) == 8) return h->Ah64;
    else if constexpr (sizeof(T) == 4) return h->Ah32;
    else return nullptr;
}

// Run restarted GMRES(m) to `tol` on (A, M = B) from x0 = 0; with Ah = A M^-1
// given (block Jacobi), each Arnoldi step is one apply of Ah.
template <int NB, typename TA, typename TB, typename TV>
static dg_status gmres_run(dg_handle* h, GmresWork& W, const TA* A, const TB* B, const TV* F, TV* x, int m,
                           double tol, int max_it, dg_solve_info* info, bool flex = false, const TA* Ah = nullptr,
                           const TV* G = nullptr) {
    const long n = (long)h->ne * NB;
    dg_status s = ensure_workspace(h, W, n, m, sizeof(TV));
    if (s != DG_OK) return s;
    if (flex && !W.Zb) {
        if ((s = dg_realloc(h, &W.Zb, (size_t)(m + 1) * W.ld * sizeof(TV))) != DG_OK) return s;
        DG_CK(h, cudaMemsetAsync(W.Zb, 0, (size_t)(m + 1) * W.ld * sizeof(TV), h->stream));
    }
    k_gm_init<TV><<<W.gx, 256, 0, h->stream>>>(F, x, (TV*)W.V, n, W.st, W.partials, m, max_it, tol);
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(W.st_host, W.st, GM_HDR, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (flex || !B || G) Ah = nullptr;
    if (flex) G = nullptr;
    // the captured cycle holds pointers, sizes and the degree: a new mesh of
    // the same size reuses it, anything else captures again
    const uintptr_t key[9] = {(uintptr_t)x, (uintptr_t)F, (uintptr_t)A, (uintptr_t)B,
                              (uintptr_t)m | ((uintptr_t)flex << 20), (uintptr_t)h->stream, (uintptr_t)Ah,
                              (uintptr_t)G, (uintptr_t)(unsigned)h->ne | ((uintptr_t)NB << 32)};
    if (W.graph && memcmp(key, W.key, sizeof(key)) != 0) {
        cudaGraphExecDestroy(W.graph);
        W.graph = nullptr;
    }
    const bool use_graph = h->stream != nullptr;  // capture needs a non-legacy stream
    if (use_graph && !W.graph && !W.st_host->done) {
        cudaGraph_t g;
        DG_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        W.nodes = enqueue_cycle<NB, TA, TB, TV>(h, W, A, B, F, x, flex, Ah, G);
        DG_CK(h, cudaStreamEndCapture(h->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&W.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return dg_cuda_fail(h, e, "cudaGraphInstantiate");
        memcpy(W.key, key, sizeof(key));
    }
    const int max_cycles = max_it + 2;
    double prev = 1.0;
    int stalls = 0;
    for (int c = 0; c < max_cycles && !W.st_host->done; ++c) {
        if (use_graph) {
            DG_CK(h, cudaGraphLaunch(W.graph, h->stream));
            h->nlaunch += W.nodes;
        } else {
            h->nlaunch += enqueue_cycle<NB, TA, TB, TV>(h, W, A, B, F, x, flex, Ah, G);
        }
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaStreamSynchronize(h->stream));
        if (flex && h->mlp.on) {
            // learned preconditioner fallback: two cycles in a row that cut the
            // true residual by less than 10% switch the correction off (block
            // Jacobi alone; FGMRES stays valid with a fixed preconditioner)
            const double rr = W.st_host->relres;
            stalls = (rr > 0.9 * prev) ? stalls + 1 : 0;
            prev = rr;
            if (stalls >= 2 && !h->mlp_fallback) {
                const int zero = 0;
                DG_CK(h, cudaMemcpyAsync(h->mlp.on, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
                h->mlp_fallback = true;
            }
        }
    }
    GmresState* hs = W.st_host;
    if (info) {
        info->iterations = hs->its;
        info->restarts = hs->cycles;
        info->outer = flex && h->mlp_fallback ? -1 : 0;
        info->relres = hs->relres;
        info->status = hs->converged ? DG_OK : DG_NOT_CONVERGED;
    }
    if (hs->nonfinite) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the GMRES iteration");
    if (!hs->converged) return dg_fail(h, DG_NOT_CONVERGED, "GMRES reached the iteration cap");
    return DG_OK;
}

template <int NB>
static dg_status gmres_f64(dg_handle* h, const double* F, double* x, dg_solve_info* info) {
    const bool mlp = h->p.precond == DG_PRECOND_MLP;
    const double* B = h->p.precond != DG_PRECOND_NONE ? h->Binv64 : nullptr;
    h->mlp_fallback = false;
    if (mlp) {
        const int one = 1;
        DG_CK(h, cudaMemcpyAsync(h->mlp.on, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    }
    const double* G = h->p.precond == DG_PRECOND_SCHWARZ ? h->G64 : nullptr;
    dg_status s = gmres_run<NB, double, double, double>(h, h->gw[0], h->A64, B, F, x, h->p.gmres_m, h->p.tol,
                                                        h->p.max_it, info, mlp, h->Ah64, G);
    if (mlp) {
        const dg_status t = dg_mlp_check_timeout(h);
        if (t != DG_OK) s = t;
    }
    if (h->gw[0].V) {
        h->basis = (const double*)h->gw[0].V;
        h->basis_ld = h->gw[0].ld;
        h->basis_n = h->gw[0].m + 1;
    }
    return s;
}

extern "C" dg_status dg_gmres_solve(dg_handle* h, const double* F, double* x, dg_solve_info* info) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "f64 blocks not stored");
    if (h->p.precond != DG_PRECOND_NONE && (!h->bj_ok || (h->p.precond == DG_PRECOND_SCHWARZ && !h->ras_ok))) {
        dg_status s = dg_precond_setup(h, h->p.precond == DG_PRECOND_SCHWARZ ? DG_PRECOND_SCHWARZ
                                                                             : DG_PRECOND_BLOCK_JACOBI);
        if (s != DG_OK) return s;
    }
    if (h->p.precond == DG_PRECOND_MLP && (!h->mlp.packed || h->mlp.nb != dg_nb(h->asm_k)))
        return dg_fail(h, DG_ERR_STATE, "MLP preconditioner: dg_mlp_init / dg_mlp_set_weights for this degree first");
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

// ---------------------------------------------------------------------------
// mixed-precision iterative refinement
// ---------------------------------------------------------------------------
// Outer loop in f64:  r = F - A64 x,  stop when ||r||/||F|| <= tol;
// inner solve in f32: A_lo d = r/||r|| by restarted GMRES(m_in) on the f32 or
// bf16 block copy with the f32 block-Jacobi inverses, to relative residual
// inner_tol;  x += ||r|| d  (f64).
struct MixState {
    double bnorm, rnorm, relres;
    unsigned int arrive;
    int first;
};

__global__ void __launch_bounds__(256) k_mx_resid(const double* __restrict__ F, const double* __restrict__ AX,
                                                   double* __restrict__ r, long n, MixState* ms, double* partials) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const double v = F[l] - AX[l];
        r[l] = v;
        a = fma(v, v, a);
    }
    const double v = dg_block_sum(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
    if (!last_block(&ms->arrive)) return;
    const double r2 = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x != 0) return;
    ms->rnorm = sqrt(r2);
    if (ms->first) {
        ms->bnorm = ms->rnorm;   // x = 0 on the first pass: r = F
        ms->first = 0;
    }
    ms->relres = ms->bnorm > 0.0 ? ms->rnorm / ms->bnorm : 0.0;
}

__global__ void __launch_bounds__(256) k_mx_scale(const double* __restrict__ r, float* __restrict__ r32, long n,
                                                   const MixState* ms) {
    const double s = ms->rnorm > 0.0 ? 1.0 / ms->rnorm : 0.0;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        r32[l] = (float)(r[l] * s);
}

__global__ void __launch_bounds__(256) k_mx_update(double* __restrict__ x, const float* __restrict__ d, long n,
                                                    const MixState* ms) {
    const double s = ms->rnorm;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        x[l] = fma(s, (double)d[l], x[l]);
}

template <int NB, typename TA>
static dg_status mixed_run(dg_handle* h, const TA* Alo, const double* F, double* x, int inner_m, double inner_tol,
                           int max_outer, dg_solve_info* info) {
    const long n = (long)h->ne * NB;
    dg_status s;
    const size_t need = (size_t)n * (8 + 8 + 4 + 4) + sizeof(MixState) + 256;
    if ((s = dg_ensure(h, &h->mx_buf, &h->cap_mx, need)) != DG_OK) return s;
    double* r64 = (double*)h->mx_buf;
    double* ax = r64 + n;
    float* r32 = (float*)(ax + n);
    float* d32 = r32 + n;
    MixState* ms = (MixState*)(((uintptr_t)(d32 + n) + 255) & ~(uintptr_t)255);
    GmresWork& W = h->gw[0];   // reuse its partials buffer for the outer reductions
    if ((s = ensure_workspace(h, W, n, h->p.gmres_m, sizeof(double))) != DG_OK) return s;
    MixState init{0.0, 0.0, 1.0, 0u, 1};
    MixState hm{};
    DG_CK(h, cudaMemcpyAsync(ms, &init, sizeof(MixState), cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));
    const bool lo16 = sizeof(TA) == 2;
    const float* B32 = (h->p.precond == DG_PRECOND_BLOCK_JACOBI || h->p.precond == DG_PRECOND_SCHWARZ)
                           ? (lo16 ? h->Binv16 : h->Binv32)
                           : nullptr;
    int inner_total = 0, outer = 0;
    const int gx = W.gx;
    bool converged = false;
    for (;;) {
        launch_apply<NB, double, double>(h, h->A64, x, ax, dctl_none(), vsel_fixed(), vsel_fixed());
        k_mx_resid<<<gx, 256, 0, h->stream>>>(F, ax, r64, n, ms, W.partials);
        h->nlaunch += 2;
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaMemcpyAsync(&hm, ms, sizeof(MixState), cudaMemcpyDeviceToHost, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
        if (!isfinite(hm.relres)) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the refinement residual");
        if (hm.relres <= h->p.tol) { converged = true; break; }
        if (outer >= max_outer || inner_total >= h->p.max_it) break;
        k_mx_scale<<<gx, 256, 0, h->stream>>>(r64, r32, n, ms);
        h->nlaunch += 1;
        DG_LAUNCH_CK(h);
        dg_solve_info in{};
        // each inner solve stops at inner_tol or after DG_INNER_CYCLES restart
        // cycles: past that the low-precision GMRES is at its accuracy floor
        // and a fresh f64 residual serves better than more inner steps
        const int cap = std::min(h->p.max_it - inner_total, DG_INNER_CYCLES * inner_m);
        s = gmres_run<NB, TA, float, float>(h, h->gw[1], Alo, B32, r32, d32, inner_m, inner_tol, cap, &in, false,
                                                ahat_of<TA>(h), h->p.precond == DG_PRECOND_SCHWARZ ? h->G32 : nullptr);
        if (s != DG_OK && s != DG_NOT_CONVERGED) return s;
        inner_total += in.iterations;
        k_mx_update<<<gx, 256, 0, h->stream>>>(x, d32, n, ms);
        h->nlaunch += 1;
        DG_LAUNCH_CK(h);
        ++outer;
    }
    if (info) {
        info->iterations = inner_total;
        info->restarts = 0;
        info->outer = outer;
        info->relres = hm.relres;
        info->status = converged ? DG_OK : DG_NOT_CONVERGED;
    }
    h->err.clear();
    if (!converged) return dg_fail(h, DG_NOT_CONVERGED, "mixed-precision refinement did not reach the tolerance");
    return DG_OK;
}

extern "C" dg_status dg_mixed_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                                    const double* F, double* x, dg_solve_info* info) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the f64 blocks are needed for the outer residual");
    if (inner_dtype != DG_F32 && inner_dtype != DG_BF16) return dg_fail(h, DG_ERR_INVALID_ARG, "inner_dtype");
    if (inner_dtype == DG_F32 && !h->A32) return dg_fail(h, DG_ERR_STATE, "f32 blocks not stored");
    if (inner_dtype == DG_BF16 && !h->A16) return dg_fail(h, DG_ERR_STATE, "bf16 blocks not stored");
    if (inner_m < 1 || inner_m > DG_MAXM || !(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
        return dg_fail(h, DG_ERR_INVALID_ARG, "inner_m / inner_tol / max_outer");
    if (h->p.precond == DG_PRECOND_BLOCK_JACOBI && !h->bj_ok) {
        dg_status s = dg_precond_setup(h, DG_PRECOND_BLOCK_JACOBI);
        if (s != DG_OK) return s;
    }
    if (h->p.precond == DG_PRECOND_SCHWARZ && !h->ras_ok) {
        dg_status s = dg_precond_setup(h, DG_PRECOND_SCHWARZ);
        if (s != DG_OK) return s;
    }
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    if (!dg_aligned16(F) || !dg_aligned16(x)) return dg_fail(h, DG_ERR_INVALID_ARG, "F and x must be 16-byte aligned");
    const int nb = dg_nb(h->asm_k);
#define DG_MIX(NBV)                                                                                          \
    if (nb == NBV)                                                                                           \
        return inner_dtype == DG_F32                                                                         \
                   ? mixed_run<NBV, float>(h, h->A32, F, x, inner_m, inner_tol, max_outer, info)             \
                   : mixed_run<NBV, __nv_bfloat16>(h, h->A16, F, x, inner_m, inner_tol, max_outer, info);
    DG_MIX(3)
    DG_MIX(6)
    DG_MIX(10)
#undef DG_MIX
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

// ---------------------------------------------------------------------------
// GMRES-based refinement: f64 flexible GMRES on A64 whose preconditioner is
// the low-precision inner solve (three-precision refinement in the sense of
// Carson & Higham): z_j = s_j A_lo^-1 V_j, with A_lo^-1 the f32 GMRES(inner_m)
// on the f32 / bf16 blocks to inner_tol or DG_INNER_CYCLES cycles.  Unlike
// plain refinement it converges when cond(A) u_lo is near or above 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ir_down(const double* __restrict__ v, float* __restrict__ r, long n) {
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        r[l] = (float)v[l];
}

__global__ void __launch_bounds__(256) k_ir_up(const float* __restrict__ d, double* __restrict__ z, long n,
                                                const double* __restrict__ scale) {
    const double s = *scale;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        z[l] = s * (double)d[l];
}

template <int NB, typename TA>
static dg_status gmres_ir_run(dg_handle* h, const TA* Alo, const double* F, double* x, int inner_m, double inner_tol,
                              int max_outer, dg_solve_info* info) {
    const long n = (long)h->ne * NB;
    const int m = h->p.gmres_m;
    GmresWork& W = h->gw[0];
    dg_status s = ensure_workspace(h, W, n, m, sizeof(double));
    if (s != DG_OK) return s;
    if (!W.Zb) {
        if ((s = dg_realloc(h, &W.Zb, (size_t)(m + 1) * W.ld * sizeof(double))) != DG_OK) return s;
        DG_CK(h, cudaMemsetAsync(W.Zb, 0, (size_t)(m + 1) * W.ld * sizeof(double), h->stream));
    }
    const size_t ld = W.ld;
    const size_t need = 2 * ld * sizeof(float) + 256;
    if ((s = dg_ensure(h, &h->mx_buf, &h->cap_mx, need)) != DG_OK) return s;
    float* r32 = (float*)h->mx_buf;
    float* d32 = r32 + ld;
    DG_CK(h, cudaMemsetAsync(h->mx_buf, 0, need, h->stream));
    const bool lo16 = sizeof(TA) == 2;
    const float* B32 = (h->p.precond == DG_PRECOND_BLOCK_JACOBI || h->p.precond == DG_PRECOND_SCHWARZ)
                           ? (lo16 ? h->Binv16 : h->Binv32)
                           : nullptr;
    double* V = (double*)W.V;
    double* Zb = (double*)W.Zb;
    double* R = (double*)W.R;
    GmresState* st = W.st;
    GmresState* hs = W.st_host;
    const long nvec = (long)W.ld / Vec<double>::W;
    const int gx = W.gx;
    k_gm_init<double><<<gx, 256, 0, h->stream>>>(F, x, V, n, st, W.partials, m, max_outer, h->p.tol);
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(hs, st, GM_HDR, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    int inner_total = 0;
    const DevCtl act{&st->active, nullptr};
    const DevCtl pend{&st->pending, nullptr};
    while (!hs->done) {
        while (hs->active) {
            const int j = hs->j;
            if (inner_total >= h->p.max_it) break;
            // z_j = s_j A_lo^-1 V_j
            k_ir_down<<<gx, 256, 0, h->stream>>>(V + (size_t)j * ld, r32, n);
            h->nlaunch += 1;
            dg_solve_info in{};
            const int cap = std::min(h->p.max_it - inner_total, DG_INNER_CYCLES * inner_m);
            s = gmres_run<NB, TA, float, float>(h, h->gw[1], Alo, B32, r32, d32, inner_m, inner_tol, cap, &in, false,
                                                ahat_of<TA>(h), h->p.precond == DG_PRECOND_SCHWARZ ? h->G32 : nullptr);
            if (s != DG_OK && s != DG_NOT_CONVERGED) return s;
            inner_total += in.iterations;
            k_ir_up<<<gx, 256, 0, h->stream>>>(d32, Zb + (size_t)j * ld, n, st->scale + j);
            // V_{j+1} = A64 z_j, orthogonalised against V_0..V_j; Givens step
            launch_apply<NB, double, double>(h, h->A64, Zb + (size_t)j * ld, V + (size_t)(j + 1) * ld, act,
                                             vsel_fixed(), vsel_fixed());
            for (int pass = 1; pass <= 2; ++pass) {
                k_gm_dots<double><<<W.gsm, dim3(GM_TX, GM_TY), 0, h->stream>>>(V, (long)ld, nvec, st, W.partials,
                                                                               pass);
                k_gm_update<double><<<gx + 1, 256, 0, h->stream>>>(V, (long)ld, nvec, st, pass);
            }
            h->nlaunch += 6;
            DG_LAUNCH_CK(h);
            DG_CK(h, cudaMemcpyAsync(hs, st, GM_HDR, cudaMemcpyDeviceToHost, h->stream));
            DG_CK(h, cudaStreamSynchronize(h->stream));
        }
        // x += Z y; true residual; restart decision
        k_gm_solve<<<1, 256, 0, h->stream>>>(st, 1);
        k_gm_combine<double><<<gx, 256, 0, h->stream>>>(Zb, (long)ld, nvec, st, R);
        k_gm_axpy<double><<<gx, 256, 0, h->stream>>>(x, R, n, st);
        launch_apply<NB, double, double>(h, h->A64, x, R, pend, vsel_fixed(), vsel_fixed());
        k_gm_resid<double><<<gx, 256, 0, h->stream>>>(F, R, V, n, st, W.partials);
        h->nlaunch += 5;
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaMemcpyAsync(hs, st, GM_HDR, cudaMemcpyDeviceToHost, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
        if (inner_total >= h->p.max_it) break;
    }
    if (info) {
        info->iterations = inner_total;
        info->restarts = hs->cycles;
        info->outer = hs->its;
        info->relres = hs->relres;
        info->status = hs->converged ? DG_OK : DG_NOT_CONVERGED;
    }
    h->err.clear();
    if (hs->nonfinite) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the outer FGMRES");
    if (!hs->converged) return dg_fail(h, DG_NOT_CONVERGED, "GMRES-based refinement did not reach the tolerance");
    return DG_OK;
}

extern "C" dg_status dg_gmres_ir_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                                       const double* F, double* x, dg_solve_info* info) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the f64 blocks are needed for the outer FGMRES");
    if (inner_dtype != DG_F32 && inner_dtype != DG_BF16) return dg_fail(h, DG_ERR_INVALID_ARG, "inner_dtype");
    if (inner_dtype == DG_F32 && !h->A32) return dg_fail(h, DG_ERR_STATE, "f32 blocks not stored");
    if (inner_dtype == DG_BF16 && !h->A16) return dg_fail(h, DG_ERR_STATE, "bf16 blocks not stored");
    if (inner_m < 1 || inner_m > DG_MAXM || !(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
        return dg_fail(h, DG_ERR_INVALID_ARG, "inner_m / inner_tol / max_outer");
    if (h->p.precond == DG_PRECOND_MLP)
        return dg_fail(h, DG_ERR_INVALID_ARG, "the inner solve takes block Jacobi, Schwarz or none");
    if (h->p.precond == DG_PRECOND_BLOCK_JACOBI && !h->bj_ok) {
        dg_status s = dg_precond_setup(h, DG_PRECOND_BLOCK_JACOBI);
        if (s != DG_OK) return s;
    }
    if (h->p.precond == DG_PRECOND_SCHWARZ && !h->ras_ok) {
        dg_status s = dg_precond_setup(h, DG_PRECOND_SCHWARZ);
        if (s != DG_OK) return s;
    }
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    if (!dg_aligned16(F) || !dg_aligned16(x)) return dg_fail(h, DG_ERR_INVALID_ARG, "F and x must be 16-byte aligned");
    const int nb = dg_nb(h->asm_k);
#define DG_GIR(NBV)                                                                                          \
    if (nb == NBV)                                                                                           \
        return inner_dtype == DG_F32                                                                         \
                   ? gmres_ir_run<NBV, float>(h, h->A32, F, x, inner_m, inner_tol, max_outer, info)          \
                   : gmres_ir_run<NBV, __nv_bfloat16>(h, h->A16, F, x, inner_m, inner_tol, max_outer, info);
    DG_GIR(3)
    DG_GIR(6)
    DG_GIR(10)
#undef DG_GIR
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

// ---------------------------------------------------------------------------
// kernel timing (instrumentation)
// ---------------------------------------------------------------------------
// A synthetic Arnoldi state: step j active, unit scales, coefficients 1e-3.
__global__ void k_prof_state(GmresState* st, int j, int m) {
    if (threadIdx.x != 0) return;
    st->active = 1;
    st->j = j;
    st->reorth = 0;
    st->m = m;
    st->its = 0;
    st->max_it = 1 << 30;
    st->tol = 0.0;
    st->bnorm = 1.0;
    st->arrive = 0;
    st->jw = j;
    st->colready = 0;
    for (int i = 0; i <= m + 1; ++i) {
        st->scale[i] = 1.0;
        st->hcol[i] = 1e-3;
        st->coef[i] = 1e-3;
    }
    for (int i = 0; i <= m; ++i) st->g[i] = i == 0 ? 1.0 : 0.0;
    for (int i = 0; i < m; ++i) {
        st->cs[i] = 1.0;
        st->sn[i] = 0.0;
    }
}

template <typename TV>
__global__ void k_prof_fill(TV* V, size_t nv, size_t n, size_t ld) {
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < nv * ld; l += (size_t)gridDim.x * blockDim.x)
        V[l] = (l % ld) < n ? (TV)(1.0 + 1e-3 * (double)(l % 977)) : (TV)0;
}

template <int NB, typename TV>
static dg_status profile_arnoldi(dg_handle* h, int which, int j, int reps, double* avg_ms) {
    GmresWork& W = h->gw[sizeof(TV) == 8 ? 0 : 1];
    const long n = (long)h->ne * NB;
    const int m = h->p.gmres_m;
    if (j < 0 || j >= m) return dg_fail(h, DG_ERR_INVALID_ARG, "j must be in [0, gmres_m)");
    dg_status s = ensure_workspace(h, W, n, m, sizeof(TV));
    if (s != DG_OK) return s;
    k_prof_fill<TV><<<1024, 256, 0, h->stream>>>((TV*)W.V, (size_t)(m + 2), (size_t)n, W.ld);
    cudaEvent_t e0, e1;
    DG_CK(h, cudaEventCreate(&e0));
    DG_CK(h, cudaEventCreate(&e1));
    double tot = 0.0;
    for (int r = 0; r < reps; ++r) {
        k_prof_state<<<1, 32, 0, h->stream>>>(W.st, j, m);
        DG_CK(h, cudaEventRecord(e0, h->stream));
        const long nvec = (long)W.ld / Vec<TV>::W;
        if constexpr (sizeof(TV) == 4) {
            if (which == DG_PROF_DOTS)
                k_gm_dots32<<<W.gd32, GM32_THREADS, 0, h->stream>>>((const float*)W.V, (long)W.ld, nvec, W.st,
                                                                  (float2*)W.partials, 1);
            else
                k_gm_update32<<<W.gu32 + 1, 256, 0, h->stream>>>((float*)W.V, (long)W.ld, nvec, W.st, 1);
        } else {
            if (which == DG_PROF_DOTS)
                k_gm_dots<TV><<<W.gsm, dim3(GM_TX, GM_TY), 0, h->stream>>>((const TV*)W.V, (long)W.ld, nvec, W.st,
                                                                             W.partials, 1);
            else
                k_gm_update<TV><<<W.gx + 1, 256, 0, h->stream>>>((TV*)W.V, (long)W.ld, nvec, W.st, 1);
        }
        DG_CK(h, cudaEventRecord(e1, h->stream));
        DG_CK(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        DG_CK(h, cudaEventElapsedTime(&ms, e0, e1));
        tot += ms;
    }
    h->nlaunch += 3 * reps + 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *avg_ms = tot / reps;
    return DG_OK;
}

// Reads the first cnt entries of V (clean lines through L2); the store never
// happens for the positive fill pattern but keeps the loads.
template <typename TV>
__global__ void k_prof_read(const TV* __restrict__ V, size_t cnt, TV* sink) {
    TV s = (TV)0;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < cnt; l += (size_t)gridDim.x * blockDim.x)
        s += V[l];
    if (s < (TV)0) *sink = s;
}

// One operator apply y = A x (block copy `dtype`) between CUDA events, with
// x = V_0 and y = V_1 of the GMRES workspace (filled once).  Before each launch
// the rest of the basis is read, which evicts A from L2 when the basis is
// larger than L2 and, being reads, leaves no dirty lines whose write-back
// would be charged to the apply.
template <typename TV>
static dg_status profile_apply(dg_handle* h, int dtype, int reps, double* avg_ms) {
    GmresWork& W = h->gw[sizeof(TV) == 8 ? 0 : 1];
    const long n = (long)h->ne * dg_nb(h->asm_k);
    const int m = h->p.gmres_m;
    dg_status s = ensure_workspace(h, W, n, m, sizeof(TV));
    if (s != DG_OK) return s;
    cudaEvent_t e0, e1;
    DG_CK(h, cudaEventCreate(&e0));
    DG_CK(h, cudaEventCreate(&e1));
    double tot = 0.0;
    TV* V = (TV*)W.V;
    k_prof_fill<TV><<<1024, 256, 0, h->stream>>>(V, (size_t)(m + 2), (size_t)n, W.ld);
    h->nlaunch += 1;
    for (int r = 0; r < reps && s == DG_OK; ++r) {
        k_prof_read<TV><<<1024, 256, 0, h->stream>>>(V + 2 * W.ld, (size_t)m * W.ld, (TV*)W.partials);
        h->nlaunch += 1;
        DG_CK(h, cudaEventRecord(e0, h->stream));
        s = dg_launch_apply(h, dtype, V, V + W.ld);
        DG_CK(h, cudaEventRecord(e1, h->stream));
        DG_CK(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        DG_CK(h, cudaEventElapsedTime(&ms, e0, e1));
        tot += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != DG_OK) return s;
    *avg_ms = tot / reps;
    return DG_OK;
}

extern "C" dg_status dg_profile_kernel(dg_handle* h, int which, int dtype, int param, int reps, double* avg_ms) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !avg_ms || reps < 1) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (which == DG_PROF_APPLY) {
        if (dtype != DG_F64 && dtype != DG_F32 && dtype != DG_BF16) return dg_fail(h, DG_ERR_INVALID_ARG, "dtype");
        DG_CK(h, cudaSetDevice(h->device));
        return dtype == DG_F64 ? profile_apply<double>(h, dtype, reps, avg_ms)
                               : profile_apply<float>(h, dtype, reps, avg_ms);
    }
    if (which != DG_PROF_DOTS && which != DG_PROF_UPDATE) return dg_fail(h, DG_ERR_INVALID_ARG, "which");
    if (dtype != DG_F64 && dtype != DG_F32) return dg_fail(h, DG_ERR_INVALID_ARG, "dtype");
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->asm_k);
#define DG_PROF(NBV)                                                                           \
    if (nb == NBV)                                                                             \
        return dtype == DG_F64 ? profile_arnoldi<NBV, double>(h, which, param, reps, avg_ms)   \
                               : profile_arnoldi<NBV, float>(h, which, param, reps, avg_ms);
    DG_PROF(3)
    DG_PROF(6)
    DG_PROF(10)
#undef DG_PROF
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}
