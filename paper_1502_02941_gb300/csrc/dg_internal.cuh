// dg_internal.cuh -- shared internals of libdg (not part of the public ABI).
//
// Data layout in HBM (all per handle):
//   geometry  geo[G_NFIELDS][ne]  f64 SoA, one field per array, element K at
//             index K: vertex 0, Jacobian J = [x1-x0 x2-x0; y1-y0 y2-y0] of the
//             affine map from the reference triangle (0,0),(1,0),(0,1), its
//             inverse and det J (= 2|K| > 0).
//   faces     nbr/nface/ftype/bidx [3][ne] i32 SoA: face f of K joins local
//             vertices f and f+1 (mod 3); nbr = neighbour across it (-1 on the
//             boundary), nface = the neighbour's local face, ftype 0 interior /
//             1 Dirichlet / 2 Neumann, bidx = boundary-edge number or -1.
//   blocks    element-row block-ELL, 4 slots per element (slot 0 = A_KK,
//             slot 1+f = A_{K,nbr(f)}).  Entries m = i*nb + j of one block are
//             cut into chunks of W = 16/sizeof(T) values; elements are grouped
//             in tiles of 32.  Entry (K, s, m) lives at
//               (((K/32)*4 + s)*C + m/W)*32*W + (K%32)*W + m%W,  C = ceil(nb^2/W)
//             so one warp (= one tile) reads one chunk of one slot as 32
//             consecutive 16-byte vectors (512 B).  Padding is zero.
//   vectors   element-major, x[K*nb + i].
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <string>
#include <unordered_map>

#include "dg.h"

#define DG_MAXK 3
#define DG_MAXNB 10
#define DG_TILE 32
#define DG_MAXM 64
#define DG_ICOEF 10   // per-instance coefficients: eps, alpha, b[6], sigma_int, sigma_bdry

enum GeoField { G_X0 = 0, G_Y0, G_J00, G_J01, G_J10, G_J11, G_I00, G_I01, G_I10, G_I11, G_DET, G_NFIELDS };

__host__ __device__ constexpr int dg_nb(int k) { return (k + 1) * (k + 2) / 2; }

// Number of 16-byte chunks per nb x nb block for element type T.
template <typename T>
__host__ __device__ constexpr int dg_chunks(int nb) { return (nb * nb + (16 / (int)sizeof(T)) - 1) / (16 / (int)sizeof(T)); }

// Offsets (in doubles) of the reference tables of one degree k.
struct TabLayout {
    int k, nb, nq, qk, qerr;
    int vol_w, vol_r, vol_s, vol_phi, vol_dr, vol_ds;        // [qk], [qk][nb]
    int face_w, face_r, face_s, face_phi, face_dr, face_ds;   // [nq], [3][nq], [3][nq][nb]
    int err_w, err_r, err_s, err_phi;                         // [qerr], [qerr][nb]
    int ct;      // DG_NCT reference contraction matrices [nb][nb] (dg_tables.cu)
    int total;
};

// Reference contraction matrices (each [nb][nb], entry [i][j], i test, j trial):
// 10 volume (S_rr, S_rs + S_sr, S_ss, C_r1, C_rr, C_rs, C_s1, C_sr, C_ss, M),
// then per face f: E_fr, E_fs, M_f, then per face pair (f, nf): X_r, X_s, Y_r,
// Y_s, Z.  See dg_tables.cu for their definitions.
#define DG_NCT_VOL 10
#define DG_NCT_SELF 3
#define DG_NCT_CROSS 5
#define DG_NCT (DG_NCT_VOL + 3 * DG_NCT_SELF + 9 * DG_NCT_CROSS)

struct GmresState;   // device-side solver state (dg_gmres.cu)

#define DG_INNER_CYCLES 8    // restart cycles per inner solve of the mixed-precision refinement
// Second Gram-Schmidt pass when the first leaves ||w - sum h_d v_d||^2 below
// this fraction of ||w||^2, i.e. when the norm drops by more than a factor 2
// (the Daniel-Gragg-Kaufman-Stewart test with eta = 1/2).  One pass then
// leaves the new vector orthogonal to about eps / eta, and the norm from
// ||w||^2 - sum h_d^2 has a relative error of about eps / eta^2.  Measured on
// the 256x256 P2 solves (f64 GMRES(50), f32-refined and f32 GMRES-IR): the same
// iteration counts and residuals as with 0.49 (eta = 0.7), 8-14 % less time.
#define DG_REORTH_FRAC 0.25
#define DG_MLP_WIDTH 128
#define DG_MLP_NOUTP 16      // output rows of the packed last layer (nb <= 10, zero padded)
#define DG_MLP_NFEAT 8       // per-element features after the 4 nb residual entries
#define DG_FLAG_MLP_TIMEOUT 8   // int slot of h->dflag: an inference kernel gave up waiting for its MMAs

// Element-local MLP right preconditioner (dg_mlp.cu).
struct MlpState {
    int nb = 0, din = 0, dinp = 0;   // unknowns per element, input width, input width padded to 16
    long P = 0;                      // parameters
    float* theta = nullptr;          // f32 master weights (flat: W1,b1,W2,b2,W3,b3,W4,b4)
    float* wr = nullptr;             // the same rounded to bf16 (values used by training)
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    int step = 0;
    bool ready = false;
    __nv_bfloat16* wbf = nullptr;    // packed inference weights W1p|W2p|W3p|W4p
    float* bias = nullptr;           // packed biases b1|b2|b3|b4p
    bool packed = false;
    float* X = nullptr;              // training rows [cap][din]
    float* T = nullptr;              // training targets [cap][nb]
    long rows = 0, cap = 0;
    float* ws = nullptr;             // training workspace
    size_t ws_cap = 0;
    int* on = nullptr;               // device flag: MLP correction enabled
    double coef[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // single-instance eps, alpha, b[6] of the last assembly
};

// Workspace of one restarted-GMRES solver instance (vectors of `elem` bytes).
struct GmresWork {
    size_t n = 0;
    size_t ld = 0;                 // leading dimension of the basis (n rounded up to 64)
    int m = 0;
    size_t elem = 0;
    void* V = nullptr;             // [(m+2)][n] Krylov basis, unnormalised
    void* Z = nullptr;             // [n] preconditioned vector / correction
    void* R = nullptr;             // [n] work vector
    void* Zb = nullptr;            // [(m+1)][ld] preconditioned directions (flexible GMRES)
    double* partials = nullptr;    // per-block reduction scratch
    GmresState* st = nullptr;      // device state
    GmresState* st_host = nullptr; // pinned mirror of the state header
    cudaGraphExec_t graph = nullptr;
    uintptr_t key[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int nodes = 0;
    int gx = 0;    // grid of the 1-D vector kernels (4 blocks of 256 per SM)
    int gsm = 0;   // grid of the multi-dot kernel (one 1024-thread block per SM)
    int gd32 = 0;  // grid of the f32 multi-dot (two 512-thread blocks per SM)
    int gu32 = 0;  // streaming blocks of the f32 update (plus its control block)
};

// A caller-supplied device buffer that the handle carves its arrays from
// (dg_set_arena): first fit over a list of free ranges, 256-byte granules,
// neighbouring free ranges merged on release.
struct DgArena {
    uintptr_t base = 0;
    size_t size = 0;
    std::map<size_t, size_t> free_ranges;         // offset -> length
    std::unordered_map<size_t, size_t> used;      // offset -> length
    void* take(size_t bytes);
    bool give_back(void* p);
};

// One live device allocation of a handle.
struct DgMemRec {
    size_t bytes;
    int cat;       // DG_WS_* category
};

struct dg_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    dg_params p{};
    bool params_set = false;

    // mesh
    int nv = 0, ne = 0, nbe = 0, nint = 0, ntiles = 0;
    bool mesh_ok = false;
    double* nodes = nullptr;
    int* elems = nullptr;
    double* geo = nullptr;
    int* nbr = nullptr;
    int* nface = nullptr;
    int* ftype = nullptr;
    int* bidx = nullptr;
    int* bedge = nullptr;          // [nbe] = 3*K + f
    double hmax = 0.0;

    // reference tables for tl.k
    double* tab = nullptr;
    TabLayout tl{};
    int tab_k = -1;

    // assembled operator
    bool assembled = false;
    int asm_k = -1;
    int asm_store = 0;
    double* A64 = nullptr;
    float* A32 = nullptr;
    __nv_bfloat16* A16 = nullptr;
    size_t A_bytes[3] = {0, 0, 0};
    double* F = nullptr;

    // block-Jacobi inverses (f64 and f32 copies), same tile layout with 1 slot
    bool bj_ok = false;
    double* Binv64 = nullptr;
    float* Binv32 = nullptr;
    float* Binv16 = nullptr;       // inverses of the bf16 diagonal blocks (f32)
    // the right-preconditioned operator A M_BJ^-1 (block-ELL, 4 slots: block
    // (K, L) = A_KL A_LL^-1, computed in f64), f64 and f32 copies: a GMRES
    // step with block Jacobi is then one apply
    double* Ah64 = nullptr;
    float* Ah32 = nullptr;
    size_t Ah_bytes[2] = {0, 0};
    // one-layer-overlap restricted additive Schwarz (DG_PRECOND_SCHWARZ): row
    // block K of the patch inverses, z_K = sum_s G_{K,s} r_{L_s} over the same
    // 4 slots as A (block-ELL), f64 and f32 copies
    bool ras_ok = false;
    double* G64 = nullptr;
    float* G32 = nullptr;
    size_t G_bytes[2] = {0, 0};

    // GMRES workspaces: [0] the f64 solver, [1] the f32 inner solver of the
    // mixed-precision refinement
    GmresWork gw[2];

    // misc scratch
    double* scratch = nullptr;
    size_t scratch_bytes = 0;
    int* dflag = nullptr;          // device error flags [8]

    // instrumentation: kernels launched by this handle (graph launches count
    // every kernel node of the graph)
    long long nlaunch = 0;

    // capacities (bytes) of arrays that are re-sized only when they must grow
    size_t cap_nodes = 0, cap_elems = 0, cap_geo = 0, cap_face = 0, cap_bedge = 0;
    size_t cap_binv64 = 0, cap_binv32 = 0, cap_binv16 = 0, cap_F = 0;

    // batch of independent instances (dg_batch.cu)
    bool b_inst_active = false;    // assembly reads per-instance coefficients
    int b_n = 0;                   // instances
    int* b_inst = nullptr;         // [ne] instance of each element
    double* b_icoef = nullptr;     // [b_n][DG_ICOEF]
    int* b_elem_start = nullptr;   // host copy [b_n+1]
    void* b_dev = nullptr;         // device solver state and tables
    size_t cap_bdev = 0;
    void* b_host = nullptr;        // pinned host mirror of per-instance results
    size_t cap_bhost = 0;
    int b_tile = 0;                // dofs per work item (autotuned)
    cudaGraphExec_t b_graph = nullptr;
    uintptr_t b_key[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int b_nodes = 0;

    MlpState mlp;
    bool mlp_fallback = false;     // the last flexible solve switched the MLP off
    bool pdl = true;               // programmatic dependent launch of the f32 Arnoldi-step kernels
    bool dense_f64 = false;        // dense solve: f64 factorization only (no f32 factors + refinement)
    bool mlp_grad_tc = false;      // dg_mlp_loss_grad on the tensor cores (as training), not the f32 GEMMs
    int nsm = 0;                   // SMs on the device
    // Krylov basis of the last f64 solve (dg_gmres_solve / dg_batch_solve with
    // DG_F64): basis_n vectors of leading dimension basis_ld (f64, unnormalised);
    // cleared when another solve starts
    const double* basis = nullptr;
    size_t basis_ld = 0;
    int basis_n = 0;

    // mixed-precision refinement buffers (r64, A x, r32, d32, state)
    void* mx_buf = nullptr;
    size_t cap_mx = 0;

    // Newton's method for the non-linear reaction (dg_nonlin.cu): the Jacobian
    // J = A + HJ in the f64 block layout, and the vectors rhs, A v, H, w
    double* J64 = nullptr;
    size_t cap_J64 = 0;
    double* nl_buf = nullptr;
    size_t cap_nl = 0;

    // device memory source and bookkeeping (dg_host.cu): cudaMalloc by
    // default, else the caller's allocator (dg_set_allocator) or a caller
    // arena (dg_set_arena); every live allocation with its size and category
    dg_alloc_fn ualloc = nullptr;
    dg_free_fn ufree = nullptr;
    void* uctx = nullptr;
    DgArena* arena = nullptr;
    std::unordered_map<void*, DgMemRec> held;
    size_t held_bytes[DG_WS_PEAK] = {0, 0, 0, 0, 0, 0, 0};   // [0] = total
    size_t peak_bytes = 0;
    int ws_cat = DG_WS_SCRATCH;    // category of allocations made now
    long fail_cuda_in = 0;         // test hook: > 0 fails the n-th checked CUDA call (DG_CK)
};

// Category of the allocations made while a scope object lives (restored on exit).
struct DgWsScope {
    dg_handle* h;
    int prev;
    DgWsScope(dg_handle* hh, int cat) : h(hh), prev(hh ? hh->ws_cat : 0) {
        if (h) h->ws_cat = cat;
    }
    ~DgWsScope() {
        if (h) h->ws_cat = prev;
    }
};
#define DG_WS_SCOPE(h, cat) DgWsScope dg_ws_scope__((h), (cat))

// error helpers (dg_host.cu)
dg_status dg_fail(dg_handle* h, dg_status s, const std::string& msg);
dg_status dg_cuda_fail(dg_handle* h, cudaError_t e, const char* what);
// Checked CUDA runtime call.  Host-side fault injection for tests: with
// DG_FAIL_CUDA_CALL=n in the environment at dg_create, the handle's n-th
// checked call reports a failure (after the real call has run and
// succeeded), so that the error path runs without any GPU fault.  Calls that
// begin or end a stream capture are not counted: failing there would leave
// the stream capturing.
static inline bool dg_injectable(const char* what) { return strstr(what, "Capture") == nullptr; }
#define DG_CK(h, call)                                                                               \
    do {                                                                                             \
        cudaError_t e__ = (call);                                                                    \
        if (e__ == cudaSuccess && (h)->fail_cuda_in > 0 && dg_injectable(#call) &&                   \
            --(h)->fail_cuda_in == 0)                                                                \
            return dg_cuda_fail((h), cudaErrorUnknown, "injected failure (DG_FAIL_CUDA_CALL) of " #call); \
        if (e__ != cudaSuccess) return dg_cuda_fail((h), e__, #call);                                \
    } while (0)
#define DG_LAUNCH_CK(h) DG_CK(h, cudaGetLastError())

// vector arguments are read with 16-byte loads
static inline bool dg_aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Device memory of a handle, from its memory source, tagged with h->ws_cat.
dg_status dg_dev_alloc(dg_handle* h, void** p, size_t bytes);
void dg_dev_free(dg_handle* h, void* p);   // NULL is accepted
// allocation helper: frees *p (if any) and allocates bytes
dg_status dg_realloc(dg_handle* h, void** p, size_t bytes);
dg_status dg_scratch(dg_handle* h, size_t bytes);   // ensure h->scratch >= bytes
// device address of the allocation-free entry point's scratch array, looked
// up at handle creation (dg_noalloc.cu)
dg_status dg_noalloc_prepare(dg_handle* h);
// DG_ERR_TIMEOUT if the learned preconditioner's kernel gave up a bounded wait
// since the last check (dg_mlp.cu); synchronises
dg_status dg_mlp_check_timeout(dg_handle* h);
// keep *p if its capacity *cap already holds bytes, else reallocate
dg_status dg_ensure(dg_handle* h, void** p, size_t* cap, size_t bytes);

// host-side table construction (dg_tables.cu)
TabLayout dg_table_layout(int k);
void dg_build_tables(int k, double* host_out);                       // host_out[layout.total]
void dg_dubiner(int k, double r, double s, double* phi, double* dr, double* ds);
void dg_gauss_legendre01(int n, double* t, double* w);
dg_status dg_ensure_tables(dg_handle* h, int k);

// launches implemented in the various translation units
dg_status dg_launch_assemble(dg_handle* h, const dg_coeffs* c, double kappa, double sig_int, double sig_bdry);
dg_status dg_launch_apply(dg_handle* h, int dtype, const void* x, void* y);
dg_status dg_launch_bj_setup(dg_handle* h);
dg_status dg_launch_bj_apply(dg_handle* h, int dtype, const void* r, void* z, const double* scale);
void dg_gmres_free(dg_handle* h, GmresWork* w);

// Launch on h->stream; with `pdl` the kernel carries the programmatic
// stream-serialisation attribute, so it may be scheduled while its predecessor
// still runs.  Such a kernel calls dg_grid_release() and then dg_grid_wait()
// before it reads anything an earlier kernel wrote, on every path.
template <typename... KArgs, typename... Args>
static inline void dg_launch_smem(dg_handle* h, bool pdl, size_t smem, void (*kern)(KArgs...), dim3 grid,
                                  dim3 block, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
}
template <typename... KArgs, typename... Args>
static inline void dg_launch(dg_handle* h, bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block,
                             Args... args) {
    dg_launch_smem(h, pdl, 0, kern, grid, block, args...);
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Programmatic dependent launch (no-ops for a kernel launched without the
// attribute): release lets the next kernel in the stream be scheduled; wait
// returns once the preceding kernel has completed and its writes are visible.
__device__ __forceinline__ void dg_grid_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void dg_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ double dg_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double dg_warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Block-wide sum; every thread gets the result.  sh must hold 32 doubles.
__device__ __forceinline__ double dg_block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = dg_warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = dg_warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// Sum of two two-float numbers (hi, lo): Knuth's TwoSum of the high parts,
// the low parts added to its error, renormalised (Dekker's fast TwoSum).  The
// compiler keeps the order of these additions (no fast-math flags).  The f32
// Krylov reductions use it across warps and blocks.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bp = s - a.x;
    float e = (a.x - (s - bp)) + (b.x - bp);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

// Index of entry (K, slot s, m) in a tile-interleaved block array of type T
// with `slots` slots per element.
template <typename T>
__host__ __device__ __forceinline__ size_t dg_blk_index(int K, int s, int m, int nb, int slots) {
    constexpr int W = 16 / (int)sizeof(T);
    const int C = dg_chunks<T>(nb);
    return ((((size_t)(K >> 5) * slots + s) * C + m / W) * 32 + (K & 31)) * W + (m % W);
}

__device__ __forceinline__ float dg_bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float dg_bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
