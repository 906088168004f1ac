// dg_batch.cu -- many independent instances of the DG problem solved together.
//
// The uploaded mesh is the concatenation of the instances' meshes (disjoint,
// each instance a contiguous range of elements), so assembly, the operator
// apply and the block-Jacobi apply run as single launches over all elements,
// with per-element instance ids selecting each instance's coefficients and
// skipping the elements of instances that are already done.  The Krylov
// reductions are segmented: the unknowns are cut into work items of `tile`
// entries that never straddle two instances; a persistent grid walks the item
// list, each item leaves one partial per dot, and the last item of an instance
// to arrive (per-instance arrival counter, no waiting) reduces that
// instance's partials in a fixed order and runs the instance's Hessenberg /
// Givens step.  All active instances take Arnoldi step j together and restart
// together every m steps; an instance that meets its tolerance drops out.
// One restart cycle is captured in a CUDA graph; the host reads the number of
// still-active instances between cycles.
//
// Mixed precision (inner_dtype DG_F32 / DG_BF16): per-instance f64 iterative
// refinement, r = F - A64 x, inner batched GMRES on f32 vectors for
// A_lo d = r/||r||, x += ||r|| d; instances whose f64 relative residual meets
// the tolerance leave the refinement.  inner_dtype DG_F64: one batched f64
// GMRES on A64 x = F.  GMRES-based refinement (dg_batch_gmres_ir_solve): a
// per-instance f64 flexible GMRES on A64 whose preconditioner is the batched
// inner solve; its state is a second solver-state set over the same items.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <type_traits>
#include <vector>

#include "dg_kernels.cuh"

template <typename TV>
dg_status dg_mlp_correct(dg_handle* h, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz, const int* iuse);

struct BState {
    int its, converged, done, reorth, pending, nonfinite, cycles, j;
    unsigned int arrive;
    int m, max_it, stalls;
    double tol, bnorm, relres, wn2_before, prevres;
    double scale[DG_MAXM + 2];
    double hcol[DG_MAXM + 2];
    double coef[DG_MAXM + 2];
    double H[(DG_MAXM + 1) * DG_MAXM];
    double cs[DG_MAXM], sn[DG_MAXM], g[DG_MAXM + 1], y[DG_MAXM];
};

// per-instance refinement state
struct BOuter {
    double bnorm, rnorm, relres, best;
    unsigned int arrive;
    int first;
    int used;   // inner Arnoldi steps spent on this instance
    int ran;    // an inner solve ran since the last residual
};

struct BatchDev {
    BState* bst;          // [nI]
    BOuter* bo;           // [nI]
    int* iactive;         // [nI] Arnoldi step active
    int* ipending;        // [nI] cycle has a correction
    int* iparticipate;    // [nI] takes part in the current inner solve
    int* iouter;          // [nI] refinement still running
    double* iscale;       // [nI] scale of the current basis vector
    int* item_inst;       // [nit]
    int* item_lo;         // [nit] first unknown
    int* item_hi;         // [nit] one past the last unknown
    int* inst_item_lo;    // [nI]
    int* inst_item_hi;    // [nI]
    double* partials;     // [nit * dots_slices][DG_MAXM+2]: per item, or per multi-dot slice
    int* jglob;           // current Arnoldi step of all active instances
    int* counters;        // [4]: active instances, nonfinite, outer-active
    int* iuse;            // [nI] learned correction still on (flexible mode), else NULL
    int nI, nit;
};

#define B_TX 32
#define B_TY 32
#define B_DPT ((DG_MAXM + 2 + B_TY - 1) / B_TY)
#define B_DOTS_SMAX 16   // most slices per work item in the multi-dots (partials per slice)

template <typename TV>
struct BAcc {
    double s = 0.0;
    __device__ __forceinline__ void fma(double a, double b) { s = ::fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct BAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void fma(float a, float b) {
        const float y = a * b - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Per-instance arrival: true in the block that processed the instance's last
// item.  Partials written before the call are visible to it (read with __ldcg).
__device__ __forceinline__ bool inst_last(unsigned int* counter, int nitems) {
    __shared__ int amlast;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int t = atomicAdd(counter, 1u);
        amlast = (t == (unsigned)nitems - 1) ? 1 : 0;
        if (amlast) *counter = 0u;
    }
    __syncthreads();
    return amlast != 0;
}

// Slice `sub` of S of work item [lo0, hi0): equal lengths rounded up to even,
// so even item bounds keep even slice bounds; the last slices may be empty.
// The updates and multi-dots split items into slices (see upd_shape and
// dots_shape) so that the blocks get even shares of the work.
__device__ __forceinline__ void b_slice(int lo0, int hi0, int S, int sub, int& lo, int& hi) {
    const int len = ((hi0 - lo0 + S - 1) / S + 1) & ~1;
    lo = min(hi0, lo0 + sub * len);
    hi = min(hi0, lo + len);
}

__device__ __forceinline__ double block_sum_1d(double v, double* sh) { return dg_block_sum(v, sh); }

// Sum partials[item][col] over the instance's items with all threads of a 1-D block.
__device__ double inst_sum(const BatchDev& B, int inst, int col, double* sh) {
    double s = 0.0;
    for (int it = B.inst_item_lo[inst] + threadIdx.x; it < B.inst_item_hi[inst]; it += blockDim.x)
        s += __ldcg(B.partials + (long)it * (DG_MAXM + 2) + col);
    return dg_block_sum(s, sh);
}

// ---------------------------------------------------------------------------
// inner batched GMRES kernels
// ---------------------------------------------------------------------------
// x = 0, V_0 = F on every item; last item of an instance: ||F||, state init.
template <typename TV>
__global__ void __launch_bounds__(256) k_b_init(const TV* __restrict__ F, TV* __restrict__ x, TV* __restrict__ V0,
                                                 BatchDev B, int m, int max_it, double tol) {
    __shared__ double sh[32];
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        double a = 0.0;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) {
            const TV f = F[l];
            x[l] = (TV)0;
            V0[l] = f;
            a = ::fma((double)f, (double)f, a);
        }
        a = dg_block_sum(a, sh);
        if (threadIdx.x == 0) B.partials[(long)it * (DG_MAXM + 2)] = a;
        if (!inst_last(&B.bst[inst].arrive, B.inst_item_hi[inst] - B.inst_item_lo[inst])) continue;
        const double b2 = inst_sum(B, inst, 0, sh);
        if (threadIdx.x == 0) {
            BState* st = B.bst + inst;
            st->m = m;
            st->max_it = max_it;
            st->tol = tol;
            st->its = 0;
            st->cycles = 0;
            st->reorth = 0;
            st->pending = 0;
            st->nonfinite = 0;
            st->j = 0;
            st->converged = 0;
            const double bn = sqrt(b2);
            st->bnorm = bn;
            st->relres = 1.0;
            int act = B.iparticipate[inst];
            if (!isfinite(bn)) {
                st->nonfinite = 1;
                act = 0;
                atomicAdd(B.counters + 1, 1);
            } else if (bn == 0.0 || tol >= 1.0) {
                st->converged = 1;
                st->relres = 0.0;
                act = 0;
            }
            st->done = act ? 0 : 1;
            st->prevres = 1.0;
            st->stalls = 0;
            B.iactive[inst] = act;
            B.ipending[inst] = 0;
            for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
            st->g[0] = bn;
            st->scale[0] = bn > 0.0 ? 1.0 / bn : 0.0;
            B.iscale[inst] = st->scale[0];
        }
        __syncthreads();
    }
}

__device__ void b_finish_column(BatchDev& B, int inst, int j, double wn, const double* hc, const double* cs,
                                const double* sn) {
    BState* st = B.bst + inst;
    const int LD = DG_MAXM + 1;
    double* Hc = st->H + (long)j * LD;
    double a = hc[0];
    for (int i = 0; i < j; ++i) {
        const double b = hc[i + 1];
        Hc[i] = cs[i] * a + sn[i] * b;
        a = -sn[i] * a + cs[i] * b;
    }
    const double r = hypot(a, wn);
    const double c = r == 0.0 ? 1.0 : a / r, s = r == 0.0 ? 0.0 : wn / r;
    st->cs[j] = c;
    st->sn[j] = s;
    Hc[j] = r;
    Hc[j + 1] = 0.0;
    const double gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->scale[j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
    B.iscale[inst] = st->scale[j + 1];
    st->its += 1;
    st->j = j + 1;
    st->pending = 1;
    B.ipending[inst] = 1;
    const bool bad = !isfinite(wn) || !isfinite(r);
    if (bad) st->nonfinite = 1;
    const double est = fabs(s * gj);
    const bool breakdown = !(wn > 1e-300) || !(r > 0.0);
    if (bad || est <= st->tol * st->bnorm || j + 1 >= st->m || st->its >= st->max_it || breakdown)
        B.iactive[inst] = 0;
}

// Segmented multi-dot: per item, r_d = <V_d, V_{j+1}> over the item's range,
// d = 0..j+1 (the last one is ||w||^2).  Last item of an instance: h_d, the
// norm ||w||^2 - sum h_d^2 and either the Givens step or a request for a
// second Gram-Schmidt pass (less than DG_REORTH_FRAC ||w||^2 left), as in
// dg_gmres.cu.
template <typename TV>
__global__ void __launch_bounds__(B_TX* B_TY) k_b_dots(const TV* __restrict__ V, long ld, BatchDev B, int pass,
                                                         int S) {
    const int j = *B.jglob;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int t = ty * B_TX + tx;
    __shared__ double hp[DG_MAXM + 2], hc[DG_MAXM + 2], css[DG_MAXM], sns[DG_MAXM];
    for (int q = blockIdx.x; q < B.nit * S; q += gridDim.x) {
        const int it = q / S;   // item; slice q - it * S of it
        const int inst = B.item_inst[it];
        BState* st = B.bst + inst;
        if (!B.iactive[inst] || (pass == 2 && !st->reorth)) continue;
        const int dlast = j + 1;
        const TV* __restrict__ w = V + (long)(j + 1) * ld;
        BAcc<TV> acc[B_DPT];
        int lo, hi;
        b_slice(B.item_lo[it], B.item_hi[it], S, q - it * S, lo, hi);
        // f64: with at most 16 dots, nsub = 32 / ncol warps share each dot (on
        // the batched workload this cut the f64 solve from 37.4 to 33.7 s, while
        // the f32 inner solves were faster without it: 12.9 against 15.7 s)
        const int ncol = dlast + 1;
        const int nsub = (sizeof(TV) == 8 && ncol <= B_TY / 2) ? B_TY / ncol : 1;
        const int dsel = nsub > 1 ? ty % ncol : ty;
        const int sub = nsub > 1 ? ty / ncol : 0;
        const bool live = ty < ncol * nsub || nsub == 1;
        for (int l = lo + tx + sub * B_TX; live && l < hi; l += B_TX * nsub) {
            const TV wl = w[l];
#pragma unroll
            for (int k = 0; k < B_DPT; ++k) {
                const int d = dsel + B_TY * k;
                if (d <= dlast) acc[k].fma(V[(long)d * ld + l], wl);
            }
        }
        if (nsub > 1) {
            const double v = dg_warp_sum(acc[0].get());
            if (tx == 0) hp[ty] = live ? v : 0.0;
            __syncthreads();
            if (t < ncol) {
                double r = 0.0;
                for (int u = 0; u < nsub; ++u) r += hp[t + u * ncol];
                B.partials[(long)q * (DG_MAXM + 2) + t] = r;
            }
            __syncthreads();
        } else {
            // only the accumulators that hold a dot are reduced (warp-uniform test)
#pragma unroll
            for (int k = 0; k < B_DPT; ++k) {
                const int d = ty + B_TY * k;
                if (d <= dlast) {
                    const double v = dg_warp_sum(acc[k].get());
                    if (tx == 0) B.partials[(long)q * (DG_MAXM + 2) + d] = v;
                }
            }
        }
        if (!inst_last(&st->arrive, (B.inst_item_hi[inst] - B.inst_item_lo[inst]) * S)) continue;
        // 16 threads per dot over the instance's items
        const int ilo = B.inst_item_lo[inst] * S, ihi = B.inst_item_hi[inst] * S;   // its slices
        for (int d0 = 0; d0 <= dlast; d0 += (B_TX * B_TY) / 16) {
            const int d = d0 + t / 16;
            double r = 0.0;
            if (d <= dlast)
                for (int i2 = ilo + t % 16; i2 < ihi; i2 += 16) r += __ldcg(B.partials + (long)i2 * (DG_MAXM + 2) + d);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if ((t % 16) == 0 && d <= dlast) {
                if (d == j + 1) {
                    hp[d] = r;
                } else {
                    const double hd = st->scale[d] * r;
                    hp[d] = hd;
                    const double h = pass == 1 ? hd : st->hcol[d] + hd;
                    st->hcol[d] = h;
                    hc[d] = h;
                    st->coef[d] = hd * st->scale[d];
                }
            }
        }
        for (int i = t; i < j; i += B_TX * B_TY) {
            css[i] = st->cs[i];
            sns[i] = st->sn[i];
        }
        __syncthreads();
        if (t == 0) {
            const double w2 = hp[j + 1];
            double s2 = 0.0;
            for (int d = 0; d <= j; ++d) s2 = ::fma(hp[d], hp[d], s2);
            const double rest = w2 - s2;
            bool ready = true;
            if (pass == 1) {
                const bool again = !(rest >= DG_REORTH_FRAC * w2);
                st->reorth = again ? 1 : 0;
                ready = !again;
            }
            if (ready) b_finish_column(B, inst, j, sqrt(rest > 0.0 ? rest : 0.0), hc, css, sns);
        }
        __syncthreads();
    }
}

// The f32 segmented multi-dot (the batched inner solves): per item the ncol
// = j+2 dots are cut into equal groups of at most 16, and the 32 warps of the
// block into (group, row partition) pairs, so every warp streams at every step
// j; lanes sum their products in f32, each warp in an f32 tree, the warps of
// a group in two-float arithmetic into the item's partial (a float2 in the
// partial's 8 bytes).  The instance's last item to arrive sums its items'
// partials in two-float and turns each dot into one f64 value: no per-warp f64
// work, which on this GPU's FP64 pipe would cost as much as the streaming.
// The tail is that of k_b_dots.
__global__ void __launch_bounds__(B_TX* B_TY) k_b_dots32(const float* __restrict__ V, long ld, BatchDev B, int pass,
                                                          int S) {
    const int j = *B.jglob;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int t = ty * B_TX + tx;
    __shared__ double hp[DG_MAXM + 2], hc[DG_MAXM + 2], css[DG_MAXM], sns[DG_MAXM];
    __shared__ float red[B_TY][16];
    __shared__ float2 tot[DG_MAXM + 2];
    const int ncol = j + 2;
    const int ngroups = (ncol + 15) / 16;
    const int gsize = (ncol + ngroups - 1) / ngroups;
    const int pb = B_TY / ngroups;
    const int g = ty % ngroups, part = ty / ngroups;
    const int d0 = g * gsize;
    const int dn = part < pb ? max(0, min(gsize, ncol - d0)) : 0;
    float2* P2 = reinterpret_cast<float2*>(B.partials);
    for (int q = blockIdx.x; q < B.nit * S; q += gridDim.x) {
        const int it = q / S;   // item; slice q - it * S of it
        const int inst = B.item_inst[it];
        BState* st = B.bst + inst;
        if (!B.iactive[inst] || (pass == 2 && !st->reorth)) continue;
        const float* __restrict__ w = V + (long)(j + 1) * ld;
        const float* __restrict__ vg = V + (long)d0 * ld;
        int lo, hi;
        b_slice(B.item_lo[it], B.item_hi[it], S, q - it * S, lo, hi);
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        if (dn > 0) {
            if (((lo | hi) & 1) == 0) {
                // even bounds (always for the split-square workloads): 8-byte slices
                for (int l = lo + 2 * (part * B_TX + tx); l < hi; l += 2 * pb * B_TX) {
                    const float2 wl = *reinterpret_cast<const float2*>(w + l);
#pragma unroll
                    for (int d = 0; d < 16; ++d)
                        if (d < dn) {
                            const float2 v = *reinterpret_cast<const float2*>(vg + (long)d * ld + l);
                            acc[d] = fmaf(v.x, wl.x, fmaf(v.y, wl.y, acc[d]));
                        }
                }
            } else {
                for (int l = lo + part * B_TX + tx; l < hi; l += pb * B_TX) {
                    const float wl = w[l];
#pragma unroll
                    for (int d = 0; d < 16; ++d)
                        if (d < dn) acc[d] = fmaf(vg[(long)d * ld + l], wl, acc[d]);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 16; ++d) {
            if (d < gsize) {   // block-uniform
                float v = acc[d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (tx == 0) red[ty][d] = d < dn ? v : 0.f;
            }
        }
        __syncthreads();
        if (t < ncol) {
            const int gg = t / gsize, dd = t - gg * gsize;
            float2 sacc = make_float2(0.f, 0.f);
            for (int p = 0; p < pb; ++p) sacc = f2_add(sacc, make_float2(red[p * ngroups + gg][dd], 0.f));
            P2[(long)q * (DG_MAXM + 2) + t] = sacc;
        }
        __syncthreads();
        if (!inst_last(&st->arrive, (B.inst_item_hi[inst] - B.inst_item_lo[inst]) * S)) continue;
        // one warp per dot over the instance's items, two-float
        const int ilo = B.inst_item_lo[inst] * S, ihi = B.inst_item_hi[inst] * S;   // its slices
        for (int d = ty; d < ncol; d += B_TY) {
            float2 sacc = make_float2(0.f, 0.f);
            for (int i2 = ilo + tx; i2 < ihi; i2 += B_TX) sacc = f2_add(sacc, __ldcg(P2 + (long)i2 * (DG_MAXM + 2) + d));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float2 q;
                q.x = __shfl_xor_sync(0xffffffffu, sacc.x, o);
                q.y = __shfl_xor_sync(0xffffffffu, sacc.y, o);
                sacc = f2_add(sacc, q);
            }
            if (tx == 0) tot[d] = sacc;
        }
        __syncthreads();
        if (t < ncol) {
            const int d = t;
            const double r = (double)tot[d].x + (double)tot[d].y;
            if (d == j + 1) {
                hp[d] = r;
            } else {
                const double hd = st->scale[d] * r;
                hp[d] = hd;
                const double h = pass == 1 ? hd : st->hcol[d] + hd;
                st->hcol[d] = h;
                hc[d] = h;
                st->coef[d] = hd * st->scale[d];
            }
        }
        for (int i = t; i < j; i += B_TX * B_TY) {
            css[i] = st->cs[i];
            sns[i] = st->sn[i];
        }
        __syncthreads();
        if (t == 0) {
            const double w2 = hp[j + 1];
            double s2 = 0.0;
            for (int d = 0; d <= j; ++d) s2 = ::fma(hp[d], hp[d], s2);
            const double rest = w2 - s2;
            bool ready = true;
            if (pass == 1) {
                const bool again = !(rest >= DG_REORTH_FRAC * w2);
                st->reorth = again ? 1 : 0;
                ready = !again;
            }
            if (ready) b_finish_column(B, inst, j, sqrt(rest > 0.0 ? rest : 0.0), hc, css, sns);
        }
        __syncthreads();
    }
}

// Segmented update: V_{j+1} -= sum_d coef_d V_d on each item (the multi-dot
// kernel already took the Givens step or asked for a second pass).

template <typename TV>
__global__ void __launch_bounds__(256) k_b_update(TV* V, long ld, BatchDev B, int pass, int S) {
    const int j = *B.jglob;
    __shared__ TV c[DG_MAXM + 2];
    for (int q = blockIdx.x; q < B.nit * S; q += gridDim.x) {
        const int it = q / S;
        int lo, hi;
        b_slice(B.item_lo[it], B.item_hi[it], S, q - it * S, lo, hi);
        const int inst = B.item_inst[it];
        BState* st = B.bst + inst;
        if (lo >= hi || !B.iactive[inst] || (pass == 2 && !st->reorth)) continue;
        __syncthreads();
        for (int d = threadIdx.x; d <= j; d += blockDim.x) c[d] = (TV)st->coef[d];
        __syncthreads();
        TV* w = V + (long)(j + 1) * ld;
        for (int l = lo + threadIdx.x; l < hi; l += blockDim.x) {
            TV acc = w[l];
            int d = 0;
            for (; d + 4 <= j + 1; d += 4) {
                const TV v0 = V[(long)d * ld + l], v1 = V[(long)(d + 1) * ld + l];
                const TV v2 = V[(long)(d + 2) * ld + l], v3 = V[(long)(d + 3) * ld + l];
                acc = ::fma(-c[d], v0, acc);
                acc = ::fma(-c[d + 1], v1, acc);
                acc = ::fma(-c[d + 2], v2, acc);
                acc = ::fma(-c[d + 3], v3, acc);
            }
            for (; d <= j; ++d) acc = ::fma(-c[d], V[(long)d * ld + l], acc);
            w[l] = acc;
        }
    }
}

// The f32 segmented update: as k_b_update, eight basis vectors in flight per
// thread and 8-byte slices where the item's bounds are even.
__global__ void __launch_bounds__(256) k_b_update32(float* V, long ld, BatchDev B, int pass, int S) {
    const int j = *B.jglob;
    __shared__ float c[DG_MAXM + 2];
    for (int q = blockIdx.x; q < B.nit * S; q += gridDim.x) {
        const int it = q / S;
        int lo, hi;
        b_slice(B.item_lo[it], B.item_hi[it], S, q - it * S, lo, hi);
        const int inst = B.item_inst[it];
        BState* st = B.bst + inst;
        if (lo >= hi || !B.iactive[inst] || (pass == 2 && !st->reorth)) continue;
        __syncthreads();
        for (int d = threadIdx.x; d <= j; d += blockDim.x) c[d] = (float)st->coef[d];
        __syncthreads();
        float* w = V + (long)(j + 1) * ld;   // aliases V: no __restrict__
        if (((lo | hi) & 1) == 0) {
            for (int l = lo + 2 * threadIdx.x; l < hi; l += 2 * blockDim.x) {
                float2 acc = *reinterpret_cast<const float2*>(w + l);
                int d = 0;
                for (; d + 8 <= j + 1; d += 8) {
                    float2 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = *reinterpret_cast<const float2*>(V + (long)(d + u) * ld + l);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        acc.x = fmaf(-c[d + u], v[u].x, acc.x);
                        acc.y = fmaf(-c[d + u], v[u].y, acc.y);
                    }
                }
                for (; d <= j; ++d) {
                    const float2 v = *reinterpret_cast<const float2*>(V + (long)d * ld + l);
                    acc.x = fmaf(-c[d], v.x, acc.x);
                    acc.y = fmaf(-c[d], v.y, acc.y);
                }
                *reinterpret_cast<float2*>(w + l) = acc;
            }
        } else {
            for (int l = lo + threadIdx.x; l < hi; l += blockDim.x) {
                float acc = w[l];
                int d = 0;
                for (; d + 8 <= j + 1; d += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = V[(long)(d + u) * ld + l];
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc = fmaf(-c[d + u], v[u], acc);
                }
                for (; d <= j; ++d) acc = fmaf(-c[d], V[(long)d * ld + l], acc);
                w[l] = acc;
            }
        }
    }
}

__global__ void k_b_step(BatchDev B) {
    if (threadIdx.x == 0) *B.jglob += 1;
}

// y = H^-1 g per pending instance (one block per instance)
__global__ void __launch_bounds__(256) k_b_solve(BatchDev B, int flexible) {
    const int inst = blockIdx.x;
    if (!B.ipending[inst]) return;
    BState* st = B.bst + inst;
    __shared__ double gs[DG_MAXM + 1];
    const int jj = st->j;
    const int LD = DG_MAXM + 1;
    for (int t = threadIdx.x; t < jj; t += blockDim.x) gs[t] = st->g[t];
    __syncthreads();
    for (int i = jj - 1; i >= 0; --i) {
        const double d = st->H[(long)i * LD + i];
        const double yi = d != 0.0 ? gs[i] / d : 0.0;
        __syncthreads();
        for (int l = threadIdx.x; l < i; l += blockDim.x) gs[l] -= st->H[(long)i * LD + l] * yi;
        if (threadIdx.x == 0) {
            st->y[i] = yi;
            st->coef[i] = flexible ? yi : yi * st->scale[i];
        }
        __syncthreads();
    }
}

// U = sum_{i<jj} coef_i V_i on the items of pending instances
template <typename TV>
__global__ void __launch_bounds__(256) k_b_combine(const TV* __restrict__ V, long ld, BatchDev B, TV* __restrict__ U) {
    __shared__ TV c[DG_MAXM + 2];
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        if (!B.ipending[inst]) continue;
        const BState* st = B.bst + inst;
        const int jj = st->j;
        __syncthreads();
        for (int d = threadIdx.x; d < jj; d += blockDim.x) c[d] = (TV)st->coef[d];
        __syncthreads();
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) {
            TV acc = (TV)0;
            for (int d = 0; d < jj; ++d) acc = ::fma(c[d], V[(long)d * ld + l], acc);
            U[l] = acc;
        }
    }
}

template <typename TV>
__global__ void __launch_bounds__(256) k_b_axpy(TV* __restrict__ x, const TV* __restrict__ z, BatchDev B) {
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        if (!B.ipending[B.item_inst[it]]) continue;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) x[l] = x[l] + z[l];
    }
}

// V_0 = F - AX on pending instances; last item: restart decision.
template <typename TV>
__global__ void __launch_bounds__(256) k_b_resid(const TV* __restrict__ F, const TV* __restrict__ AX,
                                                  TV* __restrict__ V0, BatchDev B) {
    __shared__ double sh[32];
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        if (!B.ipending[inst]) continue;
        double a = 0.0;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) {
            const TV rv = F[l] - AX[l];
            V0[l] = rv;
            a = ::fma((double)rv, (double)rv, a);
        }
        a = dg_block_sum(a, sh);
        if (threadIdx.x == 0) B.partials[(long)it * (DG_MAXM + 2)] = a;
        BState* st = B.bst + inst;
        if (!inst_last(&st->arrive, B.inst_item_hi[inst] - B.inst_item_lo[inst])) continue;
        const double r2 = inst_sum(B, inst, 0, sh);
        if (threadIdx.x == 0) {
            const double beta = sqrt(r2);
            st->pending = 0;
            B.ipending[inst] = 0;
            st->cycles += 1;
            st->relres = beta / st->bnorm;
            st->j = 0;
            int act = 1;
            if (!isfinite(beta) || st->nonfinite) {
                st->nonfinite = 1;
                atomicAdd(B.counters + 1, 1);
                act = 0;
            } else if (st->relres <= st->tol) {
                st->converged = 1;
                act = 0;
            } else if (st->its >= st->max_it) {
                act = 0;
            }
            st->done = act ? 0 : 1;
            B.iactive[inst] = act;
            if (B.iuse && B.iuse[inst]) {
                // learned preconditioner fallback per instance: two cycles in a
                // row with less than 10% residual reduction switch it off
                st->stalls = st->relres > 0.9 * st->prevres ? st->stalls + 1 : 0;
                if (st->stalls >= 2) B.iuse[inst] = 0;
            }
            st->prevres = st->relres;
            if (act) {
                for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
                st->g[0] = beta;
                st->scale[0] = 1.0 / beta;
                B.iscale[inst] = st->scale[0];
            }
        }
        __syncthreads();
    }
}

// j = 0 for the next cycle; count instances still active
__global__ void k_b_cycle_end(BatchDev B) {
    __shared__ double sh[32];
    double c = 0.0;
    for (int i = threadIdx.x; i < B.nI; i += blockDim.x) c += B.iactive[i];
    c = dg_block_sum(c, sh);
    if (threadIdx.x == 0) {
        *B.jglob = 0;
        B.counters[0] = (int)c;
    }
}

// ---------------------------------------------------------------------------
// f64 refinement kernels
// ---------------------------------------------------------------------------
// r = F - AX on instances still refining; last item: ||r||, relres, flags.
__global__ void __launch_bounds__(256) k_bo_resid(const double* __restrict__ F, const double* __restrict__ AX,
                                                   double* __restrict__ r, BatchDev B, double tol, int max_it) {
    __shared__ double sh[32];
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        if (!B.iouter[inst]) continue;
        double a = 0.0;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) {
            const double v = F[l] - AX[l];
            r[l] = v;
            a = ::fma(v, v, a);
        }
        a = dg_block_sum(a, sh);
        if (threadIdx.x == 0) B.partials[(long)it * (DG_MAXM + 2)] = a;
        BOuter* o = B.bo + inst;
        if (!inst_last(&o->arrive, B.inst_item_hi[inst] - B.inst_item_lo[inst])) continue;
        const double r2 = inst_sum(B, inst, 0, sh);
        if (threadIdx.x == 0) {
            o->rnorm = sqrt(r2);
            if (o->first) {
                o->bnorm = o->rnorm;
                o->best = 1.0;
                o->first = 0;
            }
            if (o->ran) {
                o->used += B.bst[inst].its;
                o->ran = 0;
            }
            o->relres = o->bnorm > 0.0 ? o->rnorm / o->bnorm : 0.0;
            const bool fin = isfinite(o->relres);
            if (!fin) atomicAdd(B.counters + 1, 1);
            // stop refining on convergence, an exhausted step budget, or growth
            // of the residual (the low-precision operator is too far off)
            const bool diverging = o->relres > 2.0 * o->best;
            if (o->relres < o->best) o->best = o->relres;
            const int go = (fin && o->relres > tol && o->used < max_it && !diverging) ? 1 : 0;
            B.iouter[inst] = go;
            B.iparticipate[inst] = go;
            if (go) {
                o->ran = 1;
                atomicAdd(B.counters + 2, 1);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_bo_scale(const double* __restrict__ r, float* __restrict__ r32, BatchDev B) {
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        if (!B.iouter[inst]) continue;
        const double s = 1.0 / B.bo[inst].rnorm;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) r32[l] = (float)(r[l] * s);
    }
}

__global__ void __launch_bounds__(256) k_bo_update(double* __restrict__ x, const float* __restrict__ d, BatchDev B) {
    for (int it = blockIdx.x; it < B.nit; it += gridDim.x) {
        const int inst = B.item_inst[it];
        if (!B.iouter[inst]) continue;
        const double s = B.bo[inst].rnorm;
        for (int l = B.item_lo[it] + threadIdx.x; l < B.item_hi[it]; l += blockDim.x) x[l] = ::fma(s, (double)d[l], x[l]);
    }
}

// ---------------------------------------------------------------------------
// GMRES-based refinement kernels: the outer f64 flexible GMRES lives in state
// set Bo, the inner batched low-precision GMRES in set B, over the same items
// ---------------------------------------------------------------------------
// r = s_j V_j in f32 on the instances taking outer step j (s_j their current
// basis scale); exactly those instances take part in the inner solve.
__global__ void __launch_bounds__(256) k_bir_down(const double* __restrict__ Vj, float* __restrict__ r, BatchDev Bo,
                                                   BatchDev B) {
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < Bo.nI; i += blockDim.x) B.iparticipate[i] = Bo.iactive[i];
    for (int it = blockIdx.x; it < Bo.nit; it += gridDim.x) {
        const int inst = Bo.item_inst[it];
        if (!Bo.iactive[inst]) continue;
        const double s = Bo.iscale[inst];
        for (int l = Bo.item_lo[it] + threadIdx.x; l < Bo.item_hi[it]; l += blockDim.x) r[l] = (float)(s * Vj[l]);
    }
}

// Z_j = d, the inner solution for s_j V_j, in f64
__global__ void __launch_bounds__(256) k_bir_up(const float* __restrict__ d, double* __restrict__ Zj, BatchDev Bo) {
    for (int it = blockIdx.x; it < Bo.nit; it += gridDim.x) {
        const int inst = Bo.item_inst[it];
        if (!Bo.iactive[inst]) continue;
        for (int l = Bo.item_lo[it] + threadIdx.x; l < Bo.item_hi[it]; l += blockDim.x) Zj[l] = (double)d[l];
    }
}

// Inner steps per instance; an instance that has spent max_it inner steps
// makes the current outer step its last (its restart then ends it).
__global__ void k_bir_tally(BatchDev Bo, BatchDev B, int max_it) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Bo.nI; i += gridDim.x * blockDim.x) {
        if (!Bo.iactive[i]) continue;
        BOuter* o = Bo.bo + i;
        o->used += B.bst[i].its;
        if (o->used >= max_it) Bo.bst[i].max_it = Bo.bst[i].its + 1;
    }
}

// number of instances still taking Arnoldi steps (mid-cycle)
__global__ void k_b_count(BatchDev B) {
    __shared__ double sh[32];
    double c = 0.0;
    for (int i = threadIdx.x; i < B.nI; i += blockDim.x) c += B.iactive[i];
    c = dg_block_sum(c, sh);
    if (threadIdx.x == 0) B.counters[0] = (int)c;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Item tables (shared) and one or two solver-state sets: the inner batched
// GMRES uses set 0; the GMRES-based refinement keeps its outer flexible GMRES
// in set 1 over the same items.
struct BatchSetOffsets {
    size_t bst, bo, iactive, ipending, ipart, iouter, iscale, partials, jglob, counters, iuse;
};
struct BatchHostLayout {
    size_t item_inst, item_lo, item_hi, iilo, iihi;
    BatchSetOffsets set[2];
    size_t total;
};

// Slices per item of the multi-dots (grid: one block per SM walks them): about
// 32 slices per block, so the last round of a block is a small share.
static int dots_slices(int nit, int gsm) {
    return std::max(1, std::min(B_DOTS_SMAX, (32 * gsm + nit - 1) / std::max(1, nit)));
}

static BatchHostLayout batch_layout(int nI, int nit, int nsets, int dsl) {
    BatchHostLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = (o + bytes + 255) & ~(size_t)255;
        return r;
    };
    L.item_inst = take(sizeof(int) * nit);
    L.item_lo = take(sizeof(int) * nit);
    L.item_hi = take(sizeof(int) * nit);
    L.iilo = take(sizeof(int) * nI);
    L.iihi = take(sizeof(int) * nI);
    for (int k = 0; k < nsets; ++k) {
        BatchSetOffsets& S = L.set[k];
        S.bst = take(sizeof(BState) * nI);
        S.bo = take(sizeof(BOuter) * nI);
        S.iactive = take(sizeof(int) * nI);
        S.ipending = take(sizeof(int) * nI);
        S.ipart = take(sizeof(int) * nI);
        S.iouter = take(sizeof(int) * nI);
        S.iscale = take(sizeof(double) * nI);
        S.partials = take(sizeof(double) * (size_t)nit * dsl * (DG_MAXM + 2));   // per multi-dot slice
        S.jglob = take(sizeof(int));
        S.counters = take(sizeof(int) * 4);
        S.iuse = take(sizeof(int) * nI);
    }
    L.total = o;
    return L;
}

extern "C" dg_status dg_batch_setup(dg_handle* h, int n_inst, const int* elem_start, const double* coeffs) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || n_inst < 1 || !elem_start || !coeffs) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "upload the concatenated mesh first");
    if (elem_start[0] != 0 || elem_start[n_inst] != h->ne)
        return dg_fail(h, DG_ERR_INVALID_ARG, "elem_start must run from 0 to ne");
    for (int i = 0; i < n_inst; ++i)
        if (elem_start[i + 1] <= elem_start[i]) return dg_fail(h, DG_ERR_INVALID_ARG, "empty or unordered instance");
    DG_CK(h, cudaSetDevice(h->device));
    dg_status s;
    if ((s = dg_realloc(h, (void**)&h->b_inst, sizeof(int) * h->ne)) != DG_OK) return s;
    if ((s = dg_realloc(h, (void**)&h->b_icoef, sizeof(double) * DG_ICOEF * n_inst)) != DG_OK) return s;
    std::vector<int> inst(h->ne);
    for (int i = 0; i < n_inst; ++i)
        for (int K = elem_start[i]; K < elem_start[i + 1]; ++K) inst[K] = i;
    // the instances must not touch: no face may join two instances
    std::vector<int> nbr(3 * (size_t)h->ne);
    DG_CK(h, cudaMemcpy(nbr.data(), h->nbr, sizeof(int) * 3 * (size_t)h->ne, cudaMemcpyDeviceToHost));
    for (int f = 0; f < 3; ++f)
        for (int K = 0; K < h->ne; ++K) {
            const int L = nbr[(size_t)f * h->ne + K];
            if (L >= 0 && inst[L] != inst[K]) return dg_fail(h, DG_ERR_MESH, "two instances share an edge");
        }
    // per-instance coefficients: eps, alpha, b[6] from the caller; penalties from params
    const int k = h->p.degree;
    const double sig = h->p.sigma_int > 0.0 ? h->p.sigma_int : (h->p.method == DG_NIPG ? 1.0 : 3.0 * k * (k + 1));
    const double fac = h->p.sigma_bdry_factor > 0.0 ? h->p.sigma_bdry_factor : 2.0;
    std::vector<double> ic((size_t)DG_ICOEF * n_inst);
    for (int i = 0; i < n_inst; ++i) {
        for (int t = 0; t < 8; ++t) ic[(size_t)DG_ICOEF * i + t] = coeffs[8 * i + t];
        if (!(ic[(size_t)DG_ICOEF * i] >= 0.0)) return dg_fail(h, DG_ERR_INVALID_ARG, "eps must be >= 0");
        ic[(size_t)DG_ICOEF * i + 8] = sig;
        ic[(size_t)DG_ICOEF * i + 9] = fac * sig;
    }
    DG_CK(h, cudaMemcpy(h->b_inst, inst.data(), sizeof(int) * h->ne, cudaMemcpyHostToDevice));
    DG_CK(h, cudaMemcpy(h->b_icoef, ic.data(), sizeof(double) * ic.size(), cudaMemcpyHostToDevice));
    free(h->b_elem_start);
    h->b_elem_start = (int*)malloc(sizeof(int) * (n_inst + 1));
    memcpy(h->b_elem_start, elem_start, sizeof(int) * (n_inst + 1));
    h->b_n = n_inst;
    h->b_inst_active = true;
    h->assembled = false;
    h->bj_ok = false;
    h->ras_ok = false;
    if (h->b_graph) {
        cudaGraphExecDestroy(h->b_graph);
        h->b_graph = nullptr;
    }
    return DG_OK;
}

extern "C" dg_status dg_batch_clear(dg_handle* h) {
    if (!h) return DG_ERR_INVALID_ARG;
    h->b_inst_active = false;
    h->b_n = 0;
    h->assembled = false;
    return DG_OK;
}

// Build the item list for degree nb and tile size and bind the state set(s):
// B gets set 0; B2, if given, set 1 over the same items.
static dg_status batch_tables(dg_handle* h, int nb, int tile, BatchDev& B, BatchHostLayout& L,
                              BatchDev* B2 = nullptr) {
    std::vector<int> iinst, ilo, ihi, iilo(h->b_n), iihi(h->b_n);
    for (int i = 0; i < h->b_n; ++i) {
        const long lo = (long)h->b_elem_start[i] * nb, hi = (long)h->b_elem_start[i + 1] * nb;
        iilo[i] = (int)iinst.size();
        for (long a = lo; a < hi; a += tile) {
            iinst.push_back(i);
            ilo.push_back((int)a);
            ihi.push_back((int)std::min(hi, a + (long)tile));
        }
        iihi[i] = (int)iinst.size();
    }
    const int nit = (int)iinst.size();
    L = batch_layout(h->b_n, nit, B2 ? 2 : 1, dots_slices(nit, h->nsm));   // h->nsm: the multi-dots' grid
    dg_status s;
    if ((s = dg_ensure(h, &h->b_dev, &h->cap_bdev, L.total)) != DG_OK) return s;
    char* base = (char*)h->b_dev;
    auto bind = [&](BatchDev& D, const BatchSetOffsets& S) {
        D.bst = (BState*)(base + S.bst);
        D.bo = (BOuter*)(base + S.bo);
        D.iactive = (int*)(base + S.iactive);
        D.ipending = (int*)(base + S.ipending);
        D.iparticipate = (int*)(base + S.ipart);
        D.iouter = (int*)(base + S.iouter);
        D.iscale = (double*)(base + S.iscale);
        D.item_inst = (int*)(base + L.item_inst);
        D.item_lo = (int*)(base + L.item_lo);
        D.item_hi = (int*)(base + L.item_hi);
        D.inst_item_lo = (int*)(base + L.iilo);
        D.inst_item_hi = (int*)(base + L.iihi);
        D.partials = (double*)(base + S.partials);
        D.jglob = (int*)(base + S.jglob);
        D.counters = (int*)(base + S.counters);
        D.iuse = nullptr;
        D.nI = h->b_n;
        D.nit = nit;
    };
    bind(B, L.set[0]);
    if (B2) bind(*B2, L.set[1]);
    DG_CK(h, cudaMemsetAsync(h->b_dev, 0, L.total, h->stream));
    DG_CK(h, cudaMemcpyAsync(B.item_inst, iinst.data(), sizeof(int) * nit, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemcpyAsync(B.item_lo, ilo.data(), sizeof(int) * nit, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemcpyAsync(B.item_hi, ihi.data(), sizeof(int) * nit, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemcpyAsync(B.inst_item_lo, iilo.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemcpyAsync(B.inst_item_hi, iihi.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

struct BatchRun {
    BatchDev B;
    void* V;
    void* Z;
    void* R;
    void* Zb;     // [(m+1)][ld] preconditioned directions (flexible)
    long ld;
    int m;
    int gsm, gx;
};

// Launch shape of the segmented updates: S slices per item so that there are
// at least two blocks per resident update block (4 per SM), one block per slice.
struct UpdShape {
    unsigned grid;
    int S;
};
static UpdShape upd_shape(int nit, int gx) {
    const int S = std::max(1, std::min(16, (2 * gx + nit - 1) / std::max(1, nit)));
    return UpdShape{(unsigned)std::min(std::max(1L, (long)nit * S), 65535L), S};
}

template <int NB, typename TA, typename TB, typename TV>
static int b_enqueue_cycle(dg_handle* h, const BatchRun& Rn, const TA* A, const TB* Binv, const TV* F, TV* x,
                           const TA* Ah, const TV* G) {
    const BatchDev& B = Rn.B;
    TV* V = (TV*)Rn.V;
    TV* Z = (TV*)Rn.Z;
    TV* R = (TV*)Rn.R;
    TV* Zb = (TV*)Rn.Zb;
    const bool flex = B.iuse != nullptr;
    const unsigned ge = (unsigned)((h->ne + 255) / 256);
    DevCtl step{nullptr, nullptr, h->b_inst, B.iactive, B.iscale};
    DevCtl pend{nullptr, nullptr, h->b_inst, B.ipending, nullptr};
    VecSel vj{B.jglob, 0, Rn.ld}, vj1{B.jglob, 1, Rn.ld};
    const UpdShape us = upd_shape(B.nit, Rn.gx);
    const int dsl = dots_slices(B.nit, Rn.gsm);
    int n = 0;
    for (int it = 0; it < Rn.m; ++it) {
        if (flex) {
            VecSel zj{B.jglob, 0, Rn.ld};
            k_bj_apply<NB, TB, TV, TV><<<ge, 256, 0, h->stream>>>(Binv, V, Zb, h->ne, step, vj, zj);
            dg_mlp_correct<TV>(h, V, Zb, step, vj, zj, B.iuse);
            k_apply<NB, TA, TV, TV><<<ge, 256, 0, h->stream>>>(A, h->nbr, Zb, V, h->ne,
                                                              DevCtl{nullptr, nullptr, h->b_inst, B.iactive, nullptr},
                                                              zj, vj1);
            ++n;
        } else if (G) {
            // Schwarz: Z = s_j G V_j (per-instance scales), V_{j+1} = A Z
            k_apply<NB, TV, TV, TV><<<ge, 256, 0, h->stream>>>(G, h->nbr, V, Z, h->ne, step, vj, vsel_fixed());
            k_apply<NB, TA, TV, TV><<<ge, 256, 0, h->stream>>>(A, h->nbr, Z, V, h->ne,
                                                              DevCtl{nullptr, nullptr, h->b_inst, B.iactive, nullptr},
                                                              vsel_fixed(), vj1);
        } else if (Ah) {
            // V_{j+1} = s_j (A M^-1) V_j with the precomputed operator
            k_apply<NB, TA, TV, TV, true><<<ge, 256, 0, h->stream>>>(Ah, h->nbr, V, V + Rn.ld, h->ne, step, vj,
                                                                    vj);   // unit diagonal blocks
            --n;
        } else {
            k_bj_apply<NB, TB, TV, TV><<<ge, 256, 0, h->stream>>>(Binv, V, Z, h->ne, step, vj, vsel_fixed());
            k_apply<NB, TA, TV, TV><<<ge, 256, 0, h->stream>>>(A, h->nbr, Z, V, h->ne,
                                                              DevCtl{nullptr, nullptr, h->b_inst, B.iactive, nullptr},
                                                              vsel_fixed(), vj1);
        }
        for (int pass = 1; pass <= 2; ++pass) {
            if constexpr (sizeof(TV) == 4) {
                k_b_dots32<<<Rn.gsm, dim3(B_TX, B_TY), 0, h->stream>>>((const float*)V, Rn.ld, B, pass, dsl);
                k_b_update32<<<us.grid, 256, 0, h->stream>>>((float*)V, Rn.ld, B, pass, us.S);
            } else {
                k_b_dots<TV><<<Rn.gsm, dim3(B_TX, B_TY), 0, h->stream>>>(V, Rn.ld, B, pass, dsl);
                k_b_update<TV><<<us.grid, 256, 0, h->stream>>>(V, Rn.ld, B, pass, us.S);
            }
        }
        k_b_step<<<1, 32, 0, h->stream>>>(B);
        n += 7;
    }
    k_b_solve<<<B.nI, 256, 0, h->stream>>>(B, flex ? 1 : 0);
    if (flex) {
        k_b_combine<TV><<<Rn.gx, 256, 0, h->stream>>>(Zb, Rn.ld, B, R);
        k_b_axpy<TV><<<Rn.gx, 256, 0, h->stream>>>(x, R, B);
        --n;
    } else {
        k_b_combine<TV><<<Rn.gx, 256, 0, h->stream>>>(V, Rn.ld, B, R);
        if (G)
            k_apply<NB, TV, TV, TV><<<ge, 256, 0, h->stream>>>(G, h->nbr, R, Z, h->ne, pend, vsel_fixed(), vsel_fixed());
        else
            k_bj_apply<NB, TB, TV, TV><<<ge, 256, 0, h->stream>>>(Binv, R, Z, h->ne, pend, vsel_fixed(), vsel_fixed());
        k_b_axpy<TV><<<Rn.gx, 256, 0, h->stream>>>(x, Z, B);
    }
    k_apply<NB, TA, TV, TV><<<ge, 256, 0, h->stream>>>(A, h->nbr, x, R, h->ne, pend, vsel_fixed(), vsel_fixed());
    k_b_resid<TV><<<Rn.gx, 256, 0, h->stream>>>(F, R, V, B);
    k_b_cycle_end<<<1, 1024, 0, h->stream>>>(B);
    return n + 7;
}

template <int NB, typename TA, typename TB, typename TV>
static dg_status b_gmres(dg_handle* h, BatchRun& Rn, const TA* A, const TB* Binv, const TV* F, TV* x, double tol,
                         int max_it, int* counters_host) {
    // A M^-1 precomputed by the block-Jacobi set-up (f64 / f32 copies), or
    // the Schwarz rows in the precision of the vectors
    const TA* Ah = nullptr;
    const TV* G = nullptr;
    if (h->p.precond == DG_PRECOND_SCHWARZ) {
        if constexpr (sizeof(TV) == 8) G = h->G64;
        else G = h->G32;
    } else if (Binv && Rn.B.iuse == nullptr) {
        if constexpr (sizeof(TA) == 8) Ah = h->Ah64;
        else if constexpr (sizeof(TA) == 4) Ah = h->Ah32;
    }
    const BatchDev& B = Rn.B;
    k_b_init<TV><<<Rn.gx, 256, 0, h->stream>>>(F, x, (TV*)Rn.V, B, Rn.m, max_it, tol);
    DG_CK(h, cudaMemsetAsync(B.jglob, 0, sizeof(int), h->stream));
    k_b_cycle_end<<<1, 1024, 0, h->stream>>>(B);
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    // the captured cycle holds pointers, sizes, the degree and the item count
    const uintptr_t key[12] = {(uintptr_t)A, (uintptr_t)Binv, (uintptr_t)F, (uintptr_t)x, (uintptr_t)Rn.V,
                               (uintptr_t)B.bst,
                               (uintptr_t)Rn.m | ((uintptr_t)sizeof(TV) << 16) | ((uintptr_t)(B.iuse != nullptr) << 24),
                               (uintptr_t)h->stream, (uintptr_t)Ah, (uintptr_t)G,
                               (uintptr_t)(unsigned)h->ne | ((uintptr_t)NB << 32), (uintptr_t)(unsigned)B.nit};
    if (h->b_graph && memcmp(key, h->b_key, sizeof(key)) != 0) {
        cudaGraphExecDestroy(h->b_graph);
        h->b_graph = nullptr;
    }
    const bool use_graph = h->stream != nullptr;   // capture needs a non-legacy stream
    if (use_graph && !h->b_graph) {
        cudaGraph_t g;
        DG_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->b_nodes = b_enqueue_cycle<NB, TA, TB, TV>(h, Rn, A, Binv, F, x, Ah, G);
        cudaMemcpyAsync(counters_host, B.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream);
        DG_CK(h, cudaStreamEndCapture(h->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&h->b_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return dg_cuda_fail(h, e, "cudaGraphInstantiate (batch)");
        memcpy(h->b_key, key, sizeof(key));
    }
    DG_CK(h, cudaMemcpyAsync(counters_host, B.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    const int max_cycles = max_it + 2;
    for (int c = 0; c < max_cycles && counters_host[0] > 0; ++c) {
        if (use_graph) {
            DG_CK(h, cudaGraphLaunch(h->b_graph, h->stream));
            h->nlaunch += h->b_nodes;
        } else {
            h->nlaunch += b_enqueue_cycle<NB, TA, TB, TV>(h, Rn, A, Binv, F, x, Ah, G);
            DG_CK(h, cudaMemcpyAsync(counters_host, B.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
        }
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaStreamSynchronize(h->stream));
    }
    return DG_OK;
}

template <int NB, typename TA, typename TB>
static dg_status batch_solve_t(dg_handle* h, int inner_dtype, const TA* Alo, const TB* Binv, int inner_m,
                               double inner_tol, int max_outer, const double* F, double* x, int* its_out,
                               double* relres_out, int* status_out) {
    const long n = (long)h->ne * NB;
    const long ld = (n + 63) / 64 * 64;
    BatchRun Rn{};
    BatchHostLayout L;
    const int tile = h->b_tile > 0 ? h->b_tile : 4096;
    dg_status s = batch_tables(h, NB, tile, Rn.B, L);
    if (s != DG_OK) return s;
    const bool f64 = inner_dtype == DG_F64;
    const size_t elem = f64 ? 8 : 4;
    // vectors: V (m+2) x ld, Z, R (ld); refinement: r64, ax (n f64), rin, din (ld f32)
    const bool flex = h->p.precond == DG_PRECOND_MLP;
    const int mm = f64 ? h->p.gmres_m : inner_m;
    const size_t zbytes = flex ? (size_t)(mm + 1) * ld * elem : 0;
    const size_t vbytes = ((size_t)(inner_m + 2) * ld + 2 * ld) * elem + (f64 ? 0 : (2 * n * 8 + 2 * ld * 4)) +
                          zbytes + 1024;
    if ((s = dg_ensure(h, &h->mx_buf, &h->cap_mx, vbytes)) != DG_OK) return s;
    char* vb = (char*)h->mx_buf;
    Rn.V = vb;
    Rn.Z = vb + (size_t)(inner_m + 2) * ld * elem;
    Rn.R = (char*)Rn.Z + ld * elem;
    double* r64 = (double*)((char*)Rn.R + ld * elem);
    double* ax = r64 + n;
    float* rin = (float*)(ax + n);
    float* din = rin + ld;
    Rn.Zb = f64 ? (void*)r64 : (void*)(din + ld);
    DG_CK(h, cudaMemsetAsync(h->mx_buf, 0, vbytes, h->stream));
    if (flex) {
        Rn.B.iuse = (int*)((char*)h->b_dev + L.set[0].iuse);
        std::vector<int> ones(h->b_n, 1);
        DG_CK(h, cudaMemcpyAsync(Rn.B.iuse, ones.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
        const int one = 1;
        DG_CK(h, cudaMemcpyAsync(h->mlp.on, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
    }
    Rn.ld = ld;
    Rn.m = inner_m;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    Rn.gsm = sms;
    Rn.gx = 4 * sms;
    dg_status result = DG_OK;
    if (!h->b_host) {
        DG_CK(h, cudaMallocHost(&h->b_host, 64));
        h->cap_bhost = 64;
    }
    int* cnt = (int*)h->b_host;   // pinned: the captured cycle copies the counters here
    const BatchDev& B = Rn.B;
    std::vector<BState> hst;
    std::vector<BOuter> hbo;
    int outer = 0;
    if constexpr (std::is_same<TA, double>::value) {
        // all instances take part in one batched f64 GMRES
        std::vector<int> one(h->b_n, 1);
        DG_CK(h, cudaMemcpyAsync(B.iparticipate, one.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
        s = b_gmres<NB, double, double, double>(h, Rn, Alo, Binv, F, x, h->p.tol, h->p.max_it, cnt);
        if (s != DG_OK) result = s;
        h->basis = (const double*)Rn.V;
        h->basis_ld = Rn.ld;
        h->basis_n = Rn.m + 1;
        (void)r64; (void)ax; (void)rin; (void)din; (void)inner_tol; (void)max_outer;
    } else {
        // f64 refinement around the f32 inner batched GMRES
        std::vector<BOuter> bo0(h->b_n);
        for (auto& o : bo0) o = BOuter{0.0, 0.0, 1.0, 1.0, 0u, 1, 0, 0};
        std::vector<int> one(h->b_n, 1);
        DG_CK(h, cudaMemcpyAsync(B.bo, bo0.data(), sizeof(BOuter) * h->b_n, cudaMemcpyHostToDevice, h->stream));
        DG_CK(h, cudaMemcpyAsync(B.iouter, one.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
        DG_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));
        const unsigned ge = (unsigned)((h->ne + 255) / 256);
        for (;;) {
            DevCtl oc{nullptr, nullptr, h->b_inst, B.iouter, nullptr};
            k_apply<NB, double, double, double><<<ge, 256, 0, h->stream>>>(h->A64, h->nbr, x, ax, h->ne, oc,
                                                                           vsel_fixed(), vsel_fixed());
            DG_CK(h, cudaMemsetAsync(B.counters + 2, 0, sizeof(int), h->stream));
            k_bo_resid<<<Rn.gx, 256, 0, h->stream>>>(F, ax, r64, B, h->p.tol, h->p.max_it);
            h->nlaunch += 2;
            DG_LAUNCH_CK(h);
            DG_CK(h, cudaMemcpyAsync(cnt, B.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
            DG_CK(h, cudaStreamSynchronize(h->stream));
            if (cnt[2] == 0 || outer >= max_outer) break;
            k_bo_scale<<<Rn.gx, 256, 0, h->stream>>>(r64, rin, B);
            h->nlaunch += 1;
            // inner solves stop at inner_tol or after DG_INNER_CYCLES restart cycles
            s = b_gmres<NB, TA, TB, float>(h, Rn, Alo, Binv, rin, din, inner_tol,
                                           std::min(h->p.max_it, DG_INNER_CYCLES * inner_m), cnt);
            if (s != DG_OK) {
                result = s;
                break;
            }
            k_bo_update<<<Rn.gx, 256, 0, h->stream>>>(x, din, B);
            h->nlaunch += 1;
            DG_LAUNCH_CK(h);
            ++outer;
        }
    }
    if (flex && result == DG_OK) result = dg_mlp_check_timeout(h);
    // per-instance results
    hst.resize(h->b_n);
    hbo.resize(h->b_n);
    DG_CK(h, cudaMemcpyAsync(hst.data(), B.bst, sizeof(BState) * h->b_n, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaMemcpyAsync(hbo.data(), B.bo, sizeof(BOuter) * h->b_n, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    int nconv = 0;
    for (int i = 0; i < h->b_n; ++i) {
        const double rr = f64 ? hst[i].relres : hbo[i].relres;
        const bool ok = rr <= h->p.tol;
        nconv += ok;
        if (its_out) its_out[i] = f64 ? hst[i].its : hbo[i].used;
        if (relres_out) relres_out[i] = rr;
        if (status_out) status_out[i] = ok ? DG_OK : DG_NOT_CONVERGED;
    }
    if (result != DG_OK) return result;
    if (nconv < h->b_n)
        return dg_fail(h, DG_NOT_CONVERGED, std::to_string(h->b_n - nconv) + " instances did not converge");
    return DG_OK;
}

extern "C" dg_status dg_batch_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                                    const double* F, double* x, int* its, double* relres, int* status) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->b_inst_active || h->b_n < 1) return dg_fail(h, DG_ERR_STATE, "no batch set up");
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the f64 blocks are required");
    if (inner_m < 1 || inner_m > DG_MAXM || !(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
        return dg_fail(h, DG_ERR_INVALID_ARG, "inner_m / inner_tol / max_outer");
    if (inner_dtype == DG_F32 && !h->A32) return dg_fail(h, DG_ERR_STATE, "f32 blocks not stored");
    if (inner_dtype == DG_BF16 && !h->A16) return dg_fail(h, DG_ERR_STATE, "bf16 blocks not stored");
    if (inner_dtype != DG_F64 && inner_dtype != DG_F32 && inner_dtype != DG_BF16)
        return dg_fail(h, DG_ERR_INVALID_ARG, "inner_dtype");
    if (h->p.precond != DG_PRECOND_NONE && (!h->bj_ok || (h->p.precond == DG_PRECOND_SCHWARZ && !h->ras_ok))) {
        dg_status s = dg_precond_setup(h, h->p.precond == DG_PRECOND_SCHWARZ ? DG_PRECOND_SCHWARZ
                                                                             : DG_PRECOND_BLOCK_JACOBI);
        if (s != DG_OK) return s;
    }
    if (h->p.precond == DG_PRECOND_MLP && (!h->mlp.packed || h->mlp.nb != dg_nb(h->asm_k)))
        return dg_fail(h, DG_ERR_STATE, "MLP preconditioner: dg_mlp_init / dg_mlp_set_weights for this degree first");
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    const bool pj = h->p.precond != DG_PRECOND_NONE;
    const int nb = dg_nb(h->asm_k);
#define DG_BATCH(NBV)                                                                                             \
    if (nb == NBV) {                                                                                              \
        if (inner_dtype == DG_F64)                                                                                \
            return batch_solve_t<NBV, double, double>(h, inner_dtype, h->A64, pj ? h->Binv64 : nullptr, h->p.gmres_m, \
                                                      inner_tol, max_outer, F, x, its, relres, status);           \
        if (inner_dtype == DG_F32)                                                                                \
            return batch_solve_t<NBV, float, float>(h, inner_dtype, h->A32, pj ? h->Binv32 : nullptr, inner_m,    \
                                                    inner_tol, max_outer, F, x, its, relres, status);             \
        return batch_solve_t<NBV, __nv_bfloat16, float>(h, inner_dtype, h->A16, pj ? h->Binv16 : nullptr, inner_m, \
                                                        inner_tol, max_outer, F, x, its, relres, status);         \
    }
    DG_BATCH(3)
    DG_BATCH(6)
    DG_BATCH(10)
#undef DG_BATCH
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

// GMRES-based refinement of every instance: f64 flexible GMRES(params.gmres_m)
// on A64 (state set 1) whose preconditioner is the batched low-precision
// GMRES(inner_m) (state set 0), run for all instances taking outer step j at
// once.  The outer loop is driven from the host, one outer step at a time;
// each inner solve is the captured cycle graph of b_gmres.
template <int NB, typename TA, typename TB>
static dg_status batch_ir_t(dg_handle* h, const TA* Alo, const TB* Binv, int inner_m, double inner_tol,
                            int max_outer, const double* F, double* x, int* its_out, double* relres_out,
                            int* status_out) {
    const long n = (long)h->ne * NB;
    const long ld = (n + 63) / 64 * 64;
    const int mo = h->p.gmres_m;
    BatchRun Rn{};
    BatchDev Bo{};
    BatchHostLayout L;
    const int tile = h->b_tile > 0 ? h->b_tile : 4096;
    dg_status s = batch_tables(h, NB, tile, Rn.B, L, &Bo);
    if (s != DG_OK) return s;
    // outer (f64): V (mo+2) x ld, Z (mo+1) x ld, R; inner (f32): V (inner_m+2) x ld, Z, R, r, d
    const size_t b64 = ((size_t)(mo + 2) * ld + (size_t)(mo + 1) * ld + (size_t)ld) * sizeof(double);
    const size_t b32 = ((size_t)(inner_m + 2) * ld + 4 * (size_t)ld) * sizeof(float);
    const size_t vbytes = b64 + b32 + 1024;
    if ((s = dg_ensure(h, &h->mx_buf, &h->cap_mx, vbytes)) != DG_OK) return s;
    double* Vo = (double*)h->mx_buf;
    double* Zo = Vo + (size_t)(mo + 2) * ld;
    double* Ro = Zo + (size_t)(mo + 1) * ld;
    float* v32 = (float*)(Ro + ld);
    Rn.V = v32;
    Rn.Z = v32 + (size_t)(inner_m + 2) * ld;
    Rn.R = (float*)Rn.Z + ld;
    float* r32 = (float*)Rn.R + ld;
    float* d32 = r32 + ld;
    Rn.Zb = nullptr;
    Rn.ld = ld;
    Rn.m = inner_m;
    DG_CK(h, cudaMemsetAsync(h->mx_buf, 0, vbytes, h->stream));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    Rn.gsm = sms;
    Rn.gx = 4 * sms;
    if (!h->b_host) {
        DG_CK(h, cudaMallocHost(&h->b_host, 64));
        h->cap_bhost = 64;
    }
    int* cnt = (int*)h->b_host;   // [0..3] inner counters, [8..11] outer counters (pinned)
    int* ocnt = cnt + 8;
    std::vector<int> one(h->b_n, 1);
    DG_CK(h, cudaMemcpyAsync(Bo.iparticipate, one.data(), sizeof(int) * h->b_n, cudaMemcpyHostToDevice, h->stream));
    k_b_init<double><<<Rn.gx, 256, 0, h->stream>>>(F, x, Vo, Bo, mo, max_outer, h->p.tol);
    DG_CK(h, cudaMemsetAsync(Bo.jglob, 0, sizeof(int), h->stream));
    k_b_cycle_end<<<1, 1024, 0, h->stream>>>(Bo);
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(ocnt, Bo.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    const int cap = std::min(h->p.max_it, DG_INNER_CYCLES * inner_m);
    const unsigned ge = (unsigned)((h->ne + 255) / 256);
    const unsigned gi = (unsigned)((h->b_n + 255) / 256);
    const DevCtl oact{nullptr, nullptr, h->b_inst, Bo.iactive, nullptr};
    const UpdShape uo = upd_shape(Bo.nit, Rn.gx);
    const int dslo = dots_slices(Bo.nit, Rn.gsm);
    const DevCtl opend{nullptr, nullptr, h->b_inst, Bo.ipending, nullptr};
    dg_status result = DG_OK;
    for (int cycle = 0; ocnt[0] > 0 && cycle <= max_outer + 1; ++cycle) {
        for (int j = 0; j < mo && ocnt[0] > 0; ++j) {
            // Z_j = A_lo^-1 s_j V_j (batched inner solve), V_{j+1} = A64 Z_j,
            // Gram-Schmidt and Givens step per instance
            k_bir_down<<<Rn.gx, 256, 0, h->stream>>>(Vo + (size_t)j * ld, r32, Bo, Rn.B);
            h->nlaunch += 1;
            s = b_gmres<NB, TA, TB, float>(h, Rn, Alo, Binv, r32, d32, inner_tol, cap, cnt);
            if (s != DG_OK) {
                result = s;
                break;
            }
            k_bir_up<<<Rn.gx, 256, 0, h->stream>>>(d32, Zo + (size_t)j * ld, Bo);
            k_bir_tally<<<gi, 256, 0, h->stream>>>(Bo, Rn.B, h->p.max_it);
            k_apply<NB, double, double, double><<<ge, 256, 0, h->stream>>>(
                h->A64, h->nbr, Zo + (size_t)j * ld, Vo + (size_t)(j + 1) * ld, h->ne, oact, vsel_fixed(),
                vsel_fixed());
            for (int pass = 1; pass <= 2; ++pass) {
                k_b_dots<double><<<Rn.gsm, dim3(B_TX, B_TY), 0, h->stream>>>(Vo, ld, Bo, pass, dslo);
                k_b_update<double><<<uo.grid, 256, 0, h->stream>>>(Vo, ld, Bo, pass, uo.S);
            }
            k_b_step<<<1, 32, 0, h->stream>>>(Bo);
            k_b_count<<<1, 1024, 0, h->stream>>>(Bo);
            h->nlaunch += 10;
            DG_LAUNCH_CK(h);
            DG_CK(h, cudaMemcpyAsync(ocnt, Bo.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
            DG_CK(h, cudaStreamSynchronize(h->stream));
        }
        if (result != DG_OK) break;
        // x += Z y; true f64 residual; restart or stop per instance
        k_b_solve<<<h->b_n, 256, 0, h->stream>>>(Bo, 1);
        k_b_combine<double><<<Rn.gx, 256, 0, h->stream>>>(Zo, ld, Bo, Ro);
        k_b_axpy<double><<<Rn.gx, 256, 0, h->stream>>>(x, Ro, Bo);
        k_apply<NB, double, double, double><<<ge, 256, 0, h->stream>>>(h->A64, h->nbr, x, Ro, h->ne, opend,
                                                                       vsel_fixed(), vsel_fixed());
        k_b_resid<double><<<Rn.gx, 256, 0, h->stream>>>(F, Ro, Vo, Bo);
        k_b_cycle_end<<<1, 1024, 0, h->stream>>>(Bo);
        h->nlaunch += 6;
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaMemcpyAsync(ocnt, Bo.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
    }
    std::vector<BState> hst(h->b_n);
    std::vector<BOuter> hbo(h->b_n);
    DG_CK(h, cudaMemcpyAsync(hst.data(), Bo.bst, sizeof(BState) * h->b_n, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaMemcpyAsync(hbo.data(), Bo.bo, sizeof(BOuter) * h->b_n, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    int nconv = 0;
    for (int i = 0; i < h->b_n; ++i) {
        const bool ok = hst[i].converged && hst[i].relres <= h->p.tol;
        nconv += ok;
        if (its_out) its_out[i] = hbo[i].used;
        if (relres_out) relres_out[i] = hst[i].relres;
        if (status_out) status_out[i] = ok ? DG_OK : DG_NOT_CONVERGED;
    }
    if (result != DG_OK) return result;
    if (ocnt[1] > 0) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the batched outer FGMRES");
    if (nconv < h->b_n)
        return dg_fail(h, DG_NOT_CONVERGED, std::to_string(h->b_n - nconv) + " instances did not converge");
    return DG_OK;
}

extern "C" dg_status dg_batch_gmres_ir_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol,
                                             int max_outer, const double* F, double* x, int* its, double* relres,
                                             int* status) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->b_inst_active || h->b_n < 1) return dg_fail(h, DG_ERR_STATE, "no batch set up");
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the f64 blocks are needed for the outer FGMRES");
    if (inner_dtype != DG_F32 && inner_dtype != DG_BF16) return dg_fail(h, DG_ERR_INVALID_ARG, "inner_dtype");
    if (inner_dtype == DG_F32 && !h->A32) return dg_fail(h, DG_ERR_STATE, "f32 blocks not stored");
    if (inner_dtype == DG_BF16 && !h->A16) return dg_fail(h, DG_ERR_STATE, "bf16 blocks not stored");
    if (inner_m < 1 || inner_m > DG_MAXM || !(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
        return dg_fail(h, DG_ERR_INVALID_ARG, "inner_m / inner_tol / max_outer");
    if (h->p.precond == DG_PRECOND_MLP)
        return dg_fail(h, DG_ERR_INVALID_ARG, "the inner solve takes block Jacobi, Schwarz or none");
    if (h->p.precond != DG_PRECOND_NONE && (!h->bj_ok || (h->p.precond == DG_PRECOND_SCHWARZ && !h->ras_ok))) {
        dg_status s = dg_precond_setup(h, h->p.precond);
        if (s != DG_OK) return s;
    }
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    const bool pj = h->p.precond != DG_PRECOND_NONE;
    const int nb = dg_nb(h->asm_k);
#define DG_BIR(NBV)                                                                                           \
    if (nb == NBV)                                                                                            \
        return inner_dtype == DG_F32                                                                          \
                   ? batch_ir_t<NBV, float, float>(h, h->A32, pj ? h->Binv32 : nullptr, inner_m, inner_tol,   \
                                                   max_outer, F, x, its, relres, status)                      \
                   : batch_ir_t<NBV, __nv_bfloat16, float>(h, h->A16, pj ? h->Binv16 : nullptr, inner_m,      \
                                                           inner_tol, max_outer, F, x, its, relres, status);
    DG_BIR(3)
    DG_BIR(6)
    DG_BIR(10)
#undef DG_BIR
    return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
}

// ---------------------------------------------------------------------------
// groups of batches solved in one call
// ---------------------------------------------------------------------------
// A workload whose instances differ in degree is uploaded as one batch per
// degree (each on its own handle, with kernels specialised on the unknowns per
// element).  The group call drives every batch's solve from its own host
// thread on its handle's stream, so the batches' launch sequences run on the
// GPU at the same time and the call returns when the slowest has finished.
struct GroupJob {
    dg_handle* h;
    const double* F;
    double* x;
    int *its, *status;
    double* relres;
    dg_status result;
};

static dg_status group_run(dg_handle* const* hs, int nh, const double* const* F, double* const* x, int* const* its,
                           double* const* relres, int* const* status,
                           dg_status (*solve)(GroupJob&, const void*), const void* args) {
    if (!hs || nh < 1 || nh > 64 || !x) return DG_ERR_INVALID_ARG;
    for (int i = 0; i < nh; ++i) {
        if (!hs[i] || !x[i]) return DG_ERR_INVALID_ARG;
        for (int l = 0; l < i; ++l)
            if (hs[l] == hs[i]) return dg_fail(hs[i], DG_ERR_INVALID_ARG, "a handle appears twice in the group");
    }
    std::vector<GroupJob> jobs(nh);
    for (int i = 0; i < nh; ++i)
        jobs[i] = GroupJob{hs[i], F ? F[i] : nullptr, x[i], its ? its[i] : nullptr, status ? status[i] : nullptr,
                           relres ? relres[i] : nullptr, DG_OK};
    std::vector<std::thread> th;
    th.reserve(nh - 1);
    for (int i = 1; i < nh; ++i) th.emplace_back([&jobs, i, solve, args] { jobs[i].result = solve(jobs[i], args); });
    jobs[0].result = solve(jobs[0], args);
    for (auto& t : th) t.join();
    // the first error other than non-convergence, else non-convergence, else OK
    dg_status res = DG_OK;
    for (const GroupJob& j : jobs)
        if (j.result != DG_OK && j.result != DG_NOT_CONVERGED) return j.result;
    for (const GroupJob& j : jobs)
        if (j.result == DG_NOT_CONVERGED) res = DG_NOT_CONVERGED;
    return res;
}

struct GroupArgs {
    int inner_dtype, inner_m, max_outer;
    double inner_tol;
};

static dg_status group_solve_one(GroupJob& j, const void* a) {
    const GroupArgs& g = *(const GroupArgs*)a;
    return dg_batch_solve(j.h, g.inner_dtype, g.inner_m, g.inner_tol, g.max_outer, j.F, j.x, j.its, j.relres,
                          j.status);
}

static dg_status group_ir_one(GroupJob& j, const void* a) {
    const GroupArgs& g = *(const GroupArgs*)a;
    return dg_batch_gmres_ir_solve(j.h, g.inner_dtype, g.inner_m, g.inner_tol, g.max_outer, j.F, j.x, j.its,
                                   j.relres, j.status);
}

extern "C" dg_status dg_batch_group_solve(dg_handle* const* hs, int nh, int inner_dtype, int inner_m,
                                          double inner_tol, int max_outer, const double* const* F, double* const* x,
                                          int* const* its, double* const* relres, int* const* status) {
    const GroupArgs g{inner_dtype, inner_m, max_outer, inner_tol};
    return group_run(hs, nh, F, x, its, relres, status, group_solve_one, &g);
}

extern "C" dg_status dg_batch_group_gmres_ir_solve(dg_handle* const* hs, int nh, int inner_dtype, int inner_m,
                                                   double inner_tol, int max_outer, const double* const* F,
                                                   double* const* x, int* const* its, double* const* relres,
                                                   int* const* status) {
    const GroupArgs g{inner_dtype, inner_m, max_outer, inner_tol};
    return group_run(hs, nh, F, x, its, relres, status, group_ir_one, &g);
}

extern "C" dg_status dg_batch_set_tile(dg_handle* h, int tile) {
    if (!h || tile < 0 || (tile > 0 && (tile < 256 || tile > (1 << 20)))) return DG_ERR_INVALID_ARG;
    h->b_tile = tile;
    if (h->b_graph) {
        cudaGraphExecDestroy(h->b_graph);
        h->b_graph = nullptr;
    }
    return DG_OK;
}

// Synthetic state for timing: every instance active at step j.
__global__ void k_b_prof_state(BatchDev B, int j) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.nI; i += gridDim.x * blockDim.x) {
        BState* st = B.bst + i;
        for (int d = 0; d <= j + 1; ++d) {
            st->scale[d] = 1.0;
            st->coef[d] = 1e-3;
            st->hcol[d] = 1e-3;
        }
        st->reorth = 0;
        st->arrive = 0;
        B.iactive[i] = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.jglob = j;
}

// Choose the work-item size (unknowns per item) of the segmented reductions by
// timing the batched multi-dot on this batch for each candidate; the result is
// kept in the handle and returned through *tile.
extern "C" dg_status dg_batch_autotune(dg_handle* h, int* tile) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !tile) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    if (!h->b_inst_active || !h->assembled) return dg_fail(h, DG_ERR_STATE, "set up and assemble a batch first");
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->asm_k);
    const long n = (long)h->ne * nb;
    const long ld = (n + 63) / 64 * 64;
    const int m = 50, j = 25;
    const size_t vbytes = (size_t)(m + 2) * ld * 4 + 1024;
    dg_status s;
    if ((s = dg_ensure(h, &h->mx_buf, &h->cap_mx, vbytes)) != DG_OK) return s;
    DG_CK(h, cudaMemsetAsync(h->mx_buf, 0, vbytes, h->stream));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int cands[] = {2048, 4096, 8192, 16384, 32768};
    double best = 1e30;
    int best_tile = 4096;
    cudaEvent_t e0, e1;
    DG_CK(h, cudaEventCreate(&e0));
    DG_CK(h, cudaEventCreate(&e1));
    for (int tcand : cands) {
        BatchDev B{};
        BatchHostLayout L;
        if ((s = batch_tables(h, nb, tcand, B, L)) != DG_OK) return s;
        double tot = 0.0;
        for (int r = 0; r < 4; ++r) {
            k_b_prof_state<<<(h->b_n + 255) / 256, 256, 0, h->stream>>>(B, j);
            DG_CK(h, cudaEventRecord(e0, h->stream));
            k_b_dots32<<<sms, dim3(B_TX, B_TY), 0, h->stream>>>((const float*)h->mx_buf, ld, B, 1,
                                                                dots_slices(B.nit, sms));
            DG_CK(h, cudaEventRecord(e1, h->stream));
            DG_CK(h, cudaEventSynchronize(e1));
            float ms = 0.f;
            DG_CK(h, cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) tot += ms;
        }
        h->nlaunch += 8;
        if (tot < best) {
            best = tot;
            best_tile = tcand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->b_tile = best_tile;
    if (h->b_graph) {
        cudaGraphExecDestroy(h->b_graph);
        h->b_graph = nullptr;
    }
    *tile = best_tile;
    return DG_OK;
}
