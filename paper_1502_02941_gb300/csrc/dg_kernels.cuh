// dg_kernels.cuh -- operator-apply and block-Jacobi kernel templates shared
// by the standalone calls (dg_apply.cu) and the device-resident solvers
// (dg_gmres.cu).  See dg_apply.cu for the access pattern.
#pragma once
#include "dg_internal.cuh"

// Run-time selection of a vector inside a Krylov basis: the vector used is
// base + (*j + add) * stride when j is set, else base.
struct VecSel {
    const int* j;
    int add;
    long stride;
};
static inline VecSel vsel_fixed() { return VecSel{nullptr, 0, 0}; }
template <typename T>
__device__ __forceinline__ T* sel(T* base, const VecSel& s) {
    return s.j ? base + (long)(*s.j + s.add) * s.stride : base;
}
// Solver control seen by the kernels: `active` (exit at once when 0) and the
// basis scale factors (1/||v_i||) of lazily normalised Krylov vectors.  For a
// batch of independent instances, `inst` maps an element to its instance and
// `iactive` / `iscale` hold per-instance flags and current scale factors: an
// element of an inactive instance is skipped.
struct DevCtl {
    const int* active;
    const double* scale;
    const int* inst = nullptr;
    const int* iactive = nullptr;
    const double* iscale = nullptr;
};
static inline DevCtl dctl_none() { return DevCtl{nullptr, nullptr}; }

// Launch shape of the one-thread-per-element kernels: one warp per block when
// all of the kernel's warps can be resident at once (at most 32 blocks per
// SM), so that the blocks spread over the SMs to within one warp; 256-thread
// blocks otherwise.  A one-wave grid of 256-thread blocks leaves some SMs a
// whole extra block, which an FP64-bound kernel pays in full.
struct ElemShape {
    unsigned grid, block;
};
static inline ElemShape elem_shape(const dg_handle* h) {
    const long warps = ((long)h->ne + 31) / 32;
    if (h->nsm > 0 && warps <= 32L * h->nsm) return ElemShape{(unsigned)warps, 32u};
    return ElemShape{(unsigned)(((long)h->ne + 255) / 256), 256u};
}

// ---------------------------------------------------------------------------
// typed 16-byte chunk loads
// ---------------------------------------------------------------------------
template <typename TA, typename TACC>
struct Chunk;

template <>
struct Chunk<double, double> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void load(const double* p, double* v) {
        double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
};
template <>
struct Chunk<float, float> {
    static constexpr int W = 4;
    __device__ __forceinline__ static void load(const float* p, float* v) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};
template <>
struct Chunk<float, double> {
    static constexpr int W = 4;
    __device__ __forceinline__ static void load(const float* p, double* v) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};
template <>
struct Chunk<__nv_bfloat16, float> {
    static constexpr int W = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float* v) {
        uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        v[0] = dg_bf16_lo(t.x);
        v[1] = dg_bf16_hi(t.x);
        v[2] = dg_bf16_lo(t.y);
        v[3] = dg_bf16_hi(t.y);
        v[4] = dg_bf16_lo(t.z);
        v[5] = dg_bf16_hi(t.z);
        v[6] = dg_bf16_lo(t.w);
        v[7] = dg_bf16_hi(t.w);
    }
};

// nb consecutive vector entries of element L (read-only path).
template <int NB, typename TX, typename TACC>
__device__ __forceinline__ void load_x(const TX* __restrict__ x, int L, TACC* v) {
    const TX* p = x + (size_t)L * NB;
    if constexpr ((NB * sizeof(TX)) % 16 == 0 && sizeof(TX) == 8) {
#pragma unroll
        for (int j = 0; j < NB; j += 2) {
            double2 t = __ldg(reinterpret_cast<const double2*>(p) + j / 2);
            v[j] = t.x;
            v[j + 1] = t.y;
        }
    } else if constexpr ((NB * sizeof(TX)) % 8 == 0 && sizeof(TX) == 4) {
#pragma unroll
        for (int j = 0; j < NB; j += 2) {
            float2 t = __ldg(reinterpret_cast<const float2*>(p) + j / 2);
            v[j] = t.x;
            v[j + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = (TACC)__ldg(p + j);
    }
}

template <int NB, typename TX, typename TACC>
__device__ __forceinline__ void store_y(TX* __restrict__ y, int K, const TACC* v) {
    TX* p = y + (size_t)K * NB;
    if constexpr ((NB * sizeof(TX)) % 16 == 0 && sizeof(TX) == 8) {
#pragma unroll
        for (int j = 0; j < NB; j += 2) reinterpret_cast<double2*>(p)[j / 2] = make_double2(v[j], v[j + 1]);
    } else if constexpr ((NB * sizeof(TX)) % 8 == 0 && sizeof(TX) == 4) {
#pragma unroll
        for (int j = 0; j < NB; j += 2) reinterpret_cast<float2*>(p)[j / 2] = make_float2((float)v[j], (float)v[j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) p[j] = (TX)v[j];
    }
}

// y = A x over elements [0, ne).  nbr is [3][ne].  With a solver control
// block, the kernel exits at once when the solver is inactive and x / y are
// picked from the Krylov basis by the device-side step counter; with
// ctl.scale set, y is multiplied by the scale factor of the selected x (the
// lazily normalised basis vector; per instance through ctl.iscale in a batch).
// UNIT: slot 0 is the identity and is not read (the block-Jacobi-preconditioned
// operator A M^-1, whose diagonal blocks are A_KK A_KK^-1 = I).
template <int NB, typename TA, typename TX, typename TACC, bool UNIT = false>
__global__ void __launch_bounds__(256) k_apply(const TA* __restrict__ A, const int* __restrict__ nbr,
                                                const TX* __restrict__ x0, TX* __restrict__ y0, int ne,
                                                DevCtl ctl, VecSel sx, VecSel sy) {
    using CH = Chunk<TA, TACC>;
    constexpr int W = CH::W;
    constexpr int C = (NB * NB + W - 1) / W;
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    int Ls[4] = {K, -1, -1, -1};
    if constexpr (sizeof(TX) == 4) {
        // f32 solves launch this kernel programmatically dependent on its
        // predecessor; the adjacency is constant, so it is read before the wait
        dg_grid_release();
        if (K < ne)
#pragma unroll
            for (int f = 0; f < 3; ++f) Ls[1 + f] = __ldg(nbr + (size_t)f * ne + K);
        dg_grid_wait();
    }
    if (ctl.active && !*ctl.active) return;
    if (K >= ne) return;
    if (ctl.inst && !ctl.iactive[ctl.inst[K]]) return;
    if constexpr (sizeof(TX) != 4)
#pragma unroll
        for (int f = 0; f < 3; ++f) Ls[1 + f] = __ldg(nbr + (size_t)f * ne + K);
    const TX* __restrict__ x = sel(x0, sx);
    TX* __restrict__ y = sel(y0, sy);
    const int tile = K >> 5, lane = K & 31;
    TACC acc[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) acc[r] = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int Ln = Ls[s];
        if (Ln < 0) continue;
        TACC xv[NB];
        load_x<NB, TX, TACC>(x, Ln, xv);
        if (UNIT && s == 0) {
#pragma unroll
            for (int r = 0; r < NB; ++r) acc[r] += xv[r];
            continue;
        }
        const TA* base = A + (((size_t)tile * 4 + s) * C * 32 + lane) * W;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            TACC v[W];
            CH::load(base + (size_t)c * 32 * W, v);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int m = c * W + w;
                if (m < NB * NB) acc[m / NB] = fma(v[w], xv[m % NB], acc[m / NB]);
            }
        }
    }
    if ((ctl.scale && !ctl.inst) || (ctl.inst && ctl.iscale)) {
        const TACC sc = (TACC)(ctl.inst ? ctl.iscale[ctl.inst[K]] : ctl.scale[sx.j ? *sx.j + sx.add : 0]);
#pragma unroll
        for (int r = 0; r < NB; ++r) acc[r] *= sc;
    }
    store_y<NB, TX, TACC>(y, K, acc);
}

// z_K = scale * Binv_K r_K  (one slot, no gather).  scale = ctl.scale[sr index]
// when ctl.scale is set, else 1.  B == nullptr means no preconditioner (copy).
template <int NB, typename TA, typename TX, typename TACC>
__global__ void __launch_bounds__(256) k_bj_apply(const TA* __restrict__ B, const TX* __restrict__ r0,
                                                   TX* __restrict__ z0, int ne, DevCtl ctl, VecSel sr, VecSel sz) {
    using CH = Chunk<TA, TACC>;
    constexpr int W = CH::W;
    constexpr int C = (NB * NB + W - 1) / W;
    if constexpr (sizeof(TX) == 4) {   // programmatic dependent launch (f32 solves)
        dg_grid_release();
        dg_grid_wait();
    }
    if (ctl.active && !*ctl.active) return;
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    if (ctl.inst && !ctl.iactive[ctl.inst[K]]) return;
    const TX* __restrict__ r = sel(r0, sr);
    TX* __restrict__ z = sel(z0, sz);
    const double scale = ctl.inst ? (ctl.iscale ? ctl.iscale[ctl.inst[K]] : 1.0)
                                  : (ctl.scale ? ctl.scale[sr.j ? *sr.j + sr.add : 0] : 1.0);
    if (B == nullptr) {
        TACC v[NB];
        load_x<NB, TX, TACC>(r, K, v);
#pragma unroll
        for (int i = 0; i < NB; ++i) v[i] *= (TACC)scale;
        store_y<NB, TX, TACC>(z, K, v);
        return;
    }
    const int tile = K >> 5, lane = K & 31;
    TACC xv[NB], acc[NB];
    load_x<NB, TX, TACC>(r, K, xv);
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = 0;
    const TA* base = B + ((size_t)tile * C * 32 + lane) * W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        TACC v[W];
        CH::load(base + (size_t)c * 32 * W, v);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int m = c * W + w;
            if (m < NB * NB) acc[m / NB] = fma(v[w], xv[m % NB], acc[m / NB]);
        }
    }
    if (ctl.scale || ctl.iscale) {
        const TACC sc = (TACC)scale;
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[i] *= sc;
    }
    store_y<NB, TX, TACC>(z, K, acc);
}

