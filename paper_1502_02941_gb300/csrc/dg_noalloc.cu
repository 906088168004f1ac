// dg_noalloc.cu -- dg_l2_error_noalloc: the L2 error of dg_l2_error computed
// without allocating any device memory.
//
// Who needs it: a host program whose device memory is handed out entirely by
// another allocator (a framework's caching allocator, a fixed pool carved out
// at start-up) or a timing-critical loop that must not call cudaMalloc.  Such callers set the handle up once, then call this entry point
// as often as they like; it touches only the caller's buffers, the handle's
// existing arrays and one fixed array that lives in this library's image.
//
// The reduction scratch (one partial sum per 256-element block, plus the
// total) is the file-scope __device__ array below: 16385 doubles (128 KiB + 8 B)
// held by every GPU that loads the library until the process exits.  It bounds
// the mesh to 16384 * 256 = 4,194,304 elements; larger meshes are rejected with
// DG_ERR_INVALID_ARG before anything is launched.  Every call reuses the same
// array; each slot a call reads is written earlier in the same call, so nothing
// needs clearing, but two calls whose work overlaps on the GPU (different
// streams or handles on one device) race on it and must be serialised by the
// caller.
#include <math.h>

#include <mutex>

#include "dg_internal.cuh"

#define DG_NOALLOC_PARTIALS 16384
#define DG_NOALLOC_BLOCK 256
#define DG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double dg_noalloc_scratch[DG_NOALLOC_PARTIALS + 1];

// Device address of the array for each device ordinal, with the id of the
// CUDA context it was looked up in (in host code the symbol name is only a
// host-side stand-in).  The address is looked up when a handle is created on
// the device (dg_create calls dg_noalloc_prepare with the device current),
// which also makes the runtime load this file's module, and so allocate the
// array, at that point rather than in the first dg_l2_error_noalloc call.  A
// call whose current context differs from the one of the cached address (the
// device was reset, or its primary context released and created anew) looks
// the address up again before launching anything.
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[DG_NOALLOC_MAX_DEVICES];
static unsigned long long g_noalloc_ctx[DG_NOALLOC_MAX_DEVICES];

// Id of the current CUDA context through the driver entry points the runtime
// exposes (no link against the driver library); false if unavailable.
static bool current_context_id(unsigned long long* id) {
    typedef int (*ctx_current_fn)(void**);
    typedef int (*ctx_id_fn)(void*, unsigned long long*);
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = (ctx_current_fn)f1;
            get_id = (ctx_id_fn)f2;
        }
    }
    if (!get_current || !get_id) return false;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Look the array's address up for h->device (current) unless the cached one
// belongs to the current context.
static dg_status noalloc_scratch(dg_handle* h, double** out) {
    if (h->device < 0 || h->device >= DG_NOALLOC_MAX_DEVICES)
        return dg_fail(h, DG_ERR_INVALID_ARG, "device ordinal too large for the allocation-free entry point");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long ctx = 0;
    const bool known = current_context_id(&ctx);
    if (!g_noalloc_addr[h->device] || !known || g_noalloc_ctx[h->device] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, dg_noalloc_scratch);   // h->device is current
        if (e != cudaSuccess) return dg_cuda_fail(h, e, "cudaGetSymbolAddress(dg_noalloc_scratch)");
        g_noalloc_addr[h->device] = (double*)p;
        g_noalloc_ctx[h->device] = known ? ctx : 0;
    }
    *out = g_noalloc_addr[h->device];
    return DG_OK;
}

// Set-up at handle creation (h->device current): resolve the address once.
dg_status dg_noalloc_prepare(dg_handle* h) {
    double* p = nullptr;
    return noalloc_scratch(h, &p);
}

// One element per thread: block b writes sum over its elements of
// sum_q w_q detJ (u_h(x_q) - u(x_q))^2 into partials[b].
template <int NB>
__global__ void __launch_bounds__(DG_NOALLOC_BLOCK) k_l2_noalloc(const double* __restrict__ x,
                                                                 const double* __restrict__ uex,
                                                                 const double* __restrict__ geo,
                                                                 const double* __restrict__ tab, TabLayout L,
                                                                 int ne, double* partials) {
    extern __shared__ double sm[];
    __shared__ double sh[32];
    const int qe = L.qerr;
    for (int t = threadIdx.x; t < qe * (NB + 1); t += blockDim.x)
        sm[t] = t < qe ? tab[L.err_w + t] : tab[L.err_phi + t - qe];
    __syncthreads();
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (K < ne) {
        double c[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) c[i] = x[(size_t)K * NB + i];
        for (int q = 0; q < qe; ++q) {
            double u = 0.0;
#pragma unroll
            for (int i = 0; i < NB; ++i) u += c[i] * sm[qe + q * NB + i];
            const double d = u - uex[(size_t)K * qe + q];
            e += sm[q] * d * d;
        }
        e *= geo[G_DET * (size_t)ne + K];
    }
    e = dg_block_sum(e, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = e;
}

__global__ void k_l2_noalloc_total(double* partials, int n) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = dg_block_sum(s, sh);
    if (threadIdx.x == 0) partials[DG_NOALLOC_PARTIALS] = s;
}

extern "C" dg_status dg_l2_error_noalloc(dg_handle* h, const double* x, const double* uex_q, double* l2,
                                         double* hmax) {
    if (!h || !x || !uex_q) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    const int k = h->p.degree;
    if (h->tab_k != k || !h->tab)
        return dg_fail(h, DG_ERR_STATE,
                       "reference tables for this degree are not built yet: call dg_quad_points, "
                       "dg_boundary_info or dg_assemble once first");
    if ((long long)h->ne > (long long)DG_NOALLOC_PARTIALS * DG_NOALLOC_BLOCK)
        return dg_fail(h, DG_ERR_INVALID_ARG,
                       "dg_l2_error_noalloc handles at most 4194304 elements (16384 partial sums of 256 "
                       "elements); use dg_l2_error for larger meshes");
    DG_CK(h, cudaSetDevice(h->device));
    double* part = nullptr;
    dg_status s = noalloc_scratch(h, &part);
    if (s != DG_OK) return s;
    const int blocks = (h->ne + DG_NOALLOC_BLOCK - 1) / DG_NOALLOC_BLOCK;
    const size_t smem = sizeof(double) * h->tl.qerr * (dg_nb(k) + 1);
    switch (k) {
        case 1: k_l2_noalloc<3><<<blocks, DG_NOALLOC_BLOCK, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
        case 2: k_l2_noalloc<6><<<blocks, DG_NOALLOC_BLOCK, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
        case 3: k_l2_noalloc<10><<<blocks, DG_NOALLOC_BLOCK, smem, h->stream>>>(x, uex_q, h->geo, h->tab, h->tl, h->ne, part); break;
        default: return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    k_l2_noalloc_total<<<1, 1024, 0, h->stream>>>(part, blocks);
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    double e2 = 0.0;
    DG_CK(h, cudaMemcpyAsync(&e2, part + DG_NOALLOC_PARTIALS, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (l2) *l2 = sqrt(e2);
    if (hmax) *hmax = h->hmax;
    return DG_OK;
}
