// dg_host.cu -- handle lifetime, parameters, mesh upload (device-built
// adjacency and geometry, the paper's getmesh of Sec. 2.1), point sets and
// copies out of the handle.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "dg_internal.cuh"

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
dg_status dg_fail(dg_handle* h, dg_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

dg_status dg_cuda_fail(dg_handle* h, cudaError_t e, const char* what) {
    if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return DG_ERR_NOMEM;
    return DG_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// device memory: cudaMalloc, the caller's allocator or a caller arena
// ---------------------------------------------------------------------------
static const size_t kGranule = 256;

void* DgArena::take(size_t bytes) {
    const size_t need = (bytes + kGranule - 1) / kGranule * kGranule;
    for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, len = it->second;
        free_ranges.erase(it);
        if (len > need) free_ranges[off + need] = len - need;
        used[off] = need;
        return (void*)(base + off);
    }
    return nullptr;
}

bool DgArena::give_back(void* p) {
    const size_t off = (size_t)((uintptr_t)p - base);
    auto u = used.find(off);
    if (u == used.end()) return false;
    size_t start = off, len = u->second;
    used.erase(u);
    auto nx = free_ranges.lower_bound(start);
    if (nx != free_ranges.end() && nx->first == start + len) {   // merge with the next free range
        len += nx->second;
        nx = free_ranges.erase(nx);
    }
    if (nx != free_ranges.begin()) {                              // and with the previous one
        auto pv = std::prev(nx);
        if (pv->first + pv->second == start) {
            start = pv->first;
            len += pv->second;
            free_ranges.erase(pv);
        }
    }
    free_ranges[start] = len;
    return true;
}

dg_status dg_dev_alloc(dg_handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return DG_OK;
    if (h->arena) {
        *p = h->arena->take(bytes);
        if (!*p) return dg_fail(h, DG_ERR_NOMEM, "the caller's arena has no free range of " + std::to_string(bytes) +
                                                     " bytes (dg_workspace_size(DG_WS_PEAK) sizes it)");
    } else if (h->ualloc) {
        *p = h->ualloc(h->uctx, bytes, h->device, (void*)h->stream);
        if (!*p) return dg_fail(h, DG_ERR_NOMEM, "the caller's allocator returned NULL");
        if (((uintptr_t)*p & (kGranule - 1)) != 0) {
            h->ufree(h->uctx, *p, bytes, h->device, (void*)h->stream);
            *p = nullptr;
            return dg_fail(h, DG_ERR_INVALID_ARG, "the caller's allocator returned memory not aligned to 256 bytes");
        }
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            return dg_cuda_fail(h, e, "cudaMalloc");
        }
    }
    const int cat = (h->ws_cat > 0 && h->ws_cat < DG_WS_PEAK) ? h->ws_cat : DG_WS_SCRATCH;
    h->held[*p] = DgMemRec{bytes, cat};
    h->held_bytes[cat] += bytes;
    h->held_bytes[DG_WS_TOTAL] += bytes;
    if (h->held_bytes[DG_WS_TOTAL] > h->peak_bytes) h->peak_bytes = h->held_bytes[DG_WS_TOTAL];
    return DG_OK;
}

void dg_dev_free(dg_handle* h, void* p) {
    if (!p) return;
    auto it = h->held.find(p);
    size_t bytes = 0;
    if (it != h->held.end()) {
        bytes = it->second.bytes;
        h->held_bytes[it->second.cat] -= bytes;
        h->held_bytes[DG_WS_TOTAL] -= bytes;
        h->held.erase(it);
    }
    if (h->arena) h->arena->give_back(p);
    else if (h->ufree) h->ufree(h->uctx, p, bytes, h->device, (void*)h->stream);
    else cudaFree(p);
}

dg_status dg_realloc(dg_handle* h, void** p, size_t bytes) {
    if (*p) {
        dg_dev_free(h, *p);
        *p = nullptr;
    }
    return dg_dev_alloc(h, p, bytes);
}

dg_status dg_ensure(dg_handle* h, void** p, size_t* cap, size_t bytes) {
    if (*p && *cap >= bytes) return DG_OK;
    dg_status s = dg_realloc(h, p, bytes);
    *cap = s == DG_OK ? bytes : 0;
    return s;
}

dg_status dg_scratch(dg_handle* h, size_t bytes) {
    if (h->scratch_bytes >= bytes) return DG_OK;
    DG_WS_SCOPE(h, DG_WS_SCRATCH);
    dg_status s = dg_realloc(h, (void**)&h->scratch, bytes);
    h->scratch_bytes = s == DG_OK ? bytes : 0;
    return s;
}

// Switch the memory source of a fresh handle: only the flag block may be held.
static dg_status switch_source(dg_handle* h, dg_alloc_fn a, dg_free_fn f, void* ctx, DgArena* arena) {
    if (h->held.size() > 1 || (h->held.size() == 1 && h->held.begin()->first != (void*)h->dflag)) {
        delete arena;
        return dg_fail(h, DG_ERR_STATE, "the memory source can only be set right after dg_create, before any call "
                                        "that allocates");
    }
    DG_CK(h, cudaSetDevice(h->device));
    if (h->stream) DG_CK(h, cudaStreamSynchronize(h->stream));
    dg_dev_free(h, h->dflag);
    h->dflag = nullptr;
    delete h->arena;
    h->arena = arena;
    h->ualloc = a;
    h->ufree = f;
    h->uctx = ctx;
    h->peak_bytes = 0;
    DG_WS_SCOPE(h, DG_WS_SCRATCH);
    dg_status s = dg_dev_alloc(h, (void**)&h->dflag, 64);
    if (s != DG_OK) {
        // the new source cannot give even the flag block: stay on cudaMalloc
        const std::string msg = h->err;
        delete h->arena;
        h->arena = nullptr;
        h->ualloc = nullptr;
        h->ufree = nullptr;
        h->uctx = nullptr;
        if (dg_dev_alloc(h, (void**)&h->dflag, 64) != DG_OK) return DG_ERR_NOMEM;
        DG_CK(h, cudaMemsetAsync(h->dflag, 0, 64, h->stream));
        h->err = msg + "; the handle keeps cudaMalloc";
        return s;
    }
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, 64, h->stream));
    return DG_OK;
}

extern "C" dg_status dg_set_allocator(dg_handle* h, dg_alloc_fn alloc_fn, dg_free_fn free_fn, void* ctx) {
    if (!h) return DG_ERR_INVALID_ARG;
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return dg_fail(h, DG_ERR_INVALID_ARG, "alloc_fn and free_fn are given together (both NULL: cudaMalloc)");
    return switch_source(h, alloc_fn, free_fn, ctx, nullptr);
}

extern "C" dg_status dg_set_arena(dg_handle* h, void* base, size_t bytes) {
    if (!h) return DG_ERR_INVALID_ARG;
    if (!base || ((uintptr_t)base & (kGranule - 1)) != 0 || bytes < kGranule)
        return dg_fail(h, DG_ERR_INVALID_ARG, "the arena needs a base aligned to 256 bytes and at least 256 bytes");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, base) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
        at.device != h->device) {
        cudaGetLastError();
        return dg_fail(h, DG_ERR_INVALID_ARG, "the arena must be device memory on the handle's device");
    }
    DgArena* a = new DgArena();
    a->base = (uintptr_t)base;
    a->size = bytes / kGranule * kGranule;
    a->free_ranges[0] = a->size;
    return switch_source(h, nullptr, nullptr, nullptr, a);
}

extern "C" size_t dg_workspace_size(const dg_handle* h, int what) {
    if (!h || what < 0 || what > DG_WS_PEAK) return 0;
    if (what == DG_WS_PEAK) return h->peak_bytes;
    return h->held_bytes[what];
}

static void free_all(dg_handle* h) {
    void* ptrs[] = {h->nodes, h->elems, h->geo, h->nbr, h->nface, h->ftype, h->bidx, h->bedge, h->tab,
                    h->A64, h->A32, h->A16, h->F, h->Binv64, h->Binv32, h->Binv16, h->scratch, h->dflag, h->mx_buf,
                    h->Ah64, h->Ah32, h->G64, h->G32, h->J64, h->nl_buf};
    for (void* p : ptrs) dg_dev_free(h, p);
    for (GmresWork& w : h->gw) dg_gmres_free(h, &w);
    {
        MlpState& S = h->mlp;
        for (void* p : {(void*)S.theta, (void*)S.wr, (void*)S.m, (void*)S.v, (void*)S.grad, (void*)S.wbf,
                        (void*)S.bias, (void*)S.X, (void*)S.T, (void*)S.ws, (void*)S.on})
            dg_dev_free(h, p);
    }
    for (void* p : {(void*)h->b_inst, (void*)h->b_icoef, h->b_dev}) dg_dev_free(h, p);
    if (h->b_host) cudaFreeHost(h->b_host);
    if (h->b_graph) cudaGraphExecDestroy(h->b_graph);
    free(h->b_elem_start);
    // anything left (none expected) goes back to the source too
    while (!h->held.empty()) dg_dev_free(h, h->held.begin()->first);
    delete h->arena;
    h->arena = nullptr;
}

extern "C" const char* dg_status_string(dg_status s) {
    switch (s) {
        case DG_OK: return "DG_OK";
        case DG_ERR_INVALID_ARG: return "DG_ERR_INVALID_ARG: invalid argument";
        case DG_ERR_CUDA: return "DG_ERR_CUDA: CUDA runtime error";
        case DG_NOT_CONVERGED: return "DG_NOT_CONVERGED: iteration cap reached";
        case DG_ERR_TIMEOUT: return "DG_ERR_TIMEOUT: bounded device wait expired";
        case DG_ERR_NONFINITE: return "DG_ERR_NONFINITE: NaN or Inf";
        case DG_ERR_SINGULAR_BLOCK: return "DG_ERR_SINGULAR_BLOCK: singular diagonal block";
        case DG_ERR_MESH: return "DG_ERR_MESH: invalid mesh";
        case DG_ERR_STATE: return "DG_ERR_STATE: call order violated";
        case DG_ERR_NOMEM: return "DG_ERR_NOMEM: device allocation failed";
        default: return "unknown dg_status";
    }
}

extern "C" const char* dg_last_error(const dg_handle* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" dg_status dg_params_default(dg_params* p) {
    if (!p) return DG_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->method = DG_SIPG;
    p->degree = 1;
    p->sigma_int = 0.0;
    p->sigma_bdry_factor = 2.0;
    p->b0 = 1.0;
    p->store = DG_STORE_F64;
    p->gmres_m = 50;
    p->tol = 1e-10;
    p->max_it = 10000;
    p->precond = DG_PRECOND_BLOCK_JACOBI;
    return DG_OK;
}

extern "C" dg_status dg_create(dg_handle** out, int device, void* stream) {
    if (!out) return DG_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return DG_ERR_CUDA;
    if (device < 0 || device >= ndev) return DG_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DG_ERR_CUDA;
    dg_handle* h = new dg_handle();
    h->device = device;
    h->stream = (cudaStream_t)stream;
    const char* pdl = getenv("DG_PDL");
    h->pdl = !(pdl && pdl[0] == '0');
    const char* d64 = getenv("DG_DENSE_F64");
    h->dense_f64 = d64 && d64[0] == '1';
    const char* gtc = getenv("DG_MLP_GRAD_TC");
    h->mlp_grad_tc = gtc && gtc[0] == '1';
    const char* inj = getenv("DG_FAIL_CUDA_CALL");   // test hook, see DG_CK
    h->fail_cuda_in = inj ? atol(inj) : 0;
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete h;
        return DG_ERR_CUDA;
    }
    dg_params_default(&h->p);
    if (dg_realloc(h, (void**)&h->dflag, 64) != DG_OK) {
        delete h;
        return DG_ERR_NOMEM;
    }
    if (cudaMemset(h->dflag, 0, 64) != cudaSuccess) {
        cudaFree(h->dflag);
        delete h;
        return DG_ERR_CUDA;
    }
    // the allocation-free entry point's scratch address (dg_noalloc.cu)
    if (dg_noalloc_prepare(h) != DG_OK) {
        cudaFree(h->dflag);
        delete h;
        return DG_ERR_CUDA;
    }
    *out = h;
    return DG_OK;
}

extern "C" dg_status dg_destroy(dg_handle* h) {
    if (!h) return DG_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return DG_OK;
}

extern "C" dg_status dg_set_stream(dg_handle* h, void* stream) {
    if (!h) return DG_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    for (GmresWork& w : h->gw)
        if (w.graph) {
            cudaGraphExecDestroy(w.graph);
            w.graph = nullptr;
        }
    return DG_OK;
}

extern "C" dg_status dg_set_params(dg_handle* h, const dg_params* p) {
    if (!h || !p) return DG_ERR_INVALID_ARG;
    if (p->method < DG_NIPG || p->method > DG_IIPG) return dg_fail(h, DG_ERR_INVALID_ARG, "method must be 1..3");
    if (p->degree < 1 || p->degree > DG_MAXK) return dg_fail(h, DG_ERR_INVALID_ARG, "degree must be 1..3");
    if (!(p->b0 >= 1.0 && p->b0 <= 8.0)) return dg_fail(h, DG_ERR_INVALID_ARG, "b0 must be in [1, 8]");
    if ((p->store & 7) == 0 || (p->store & ~7)) return dg_fail(h, DG_ERR_INVALID_ARG, "store mask");
    if (p->gmres_m < 1 || p->gmres_m > DG_MAXM) return dg_fail(h, DG_ERR_INVALID_ARG, "gmres_m must be 1..64");
    if (!(p->tol > 0.0) || p->max_it < 1) return dg_fail(h, DG_ERR_INVALID_ARG, "tol/max_it");
    if (p->precond != DG_PRECOND_NONE && p->precond != DG_PRECOND_BLOCK_JACOBI && p->precond != DG_PRECOND_MLP &&
        p->precond != DG_PRECOND_SCHWARZ)
        return dg_fail(h, DG_ERR_INVALID_ARG, "precond");
    if (p->degree != h->p.degree || p->store != h->p.store) {
        h->assembled = false;
        h->bj_ok = false;
        h->ras_ok = false;
    }
    h->p = *p;
    h->params_set = true;
    return DG_OK;
}

// ---------------------------------------------------------------------------
// mesh upload: device kernels
// ---------------------------------------------------------------------------
enum MeshFlag { MF_BAD_INDEX = 1, MF_CLOCKWISE = 2, MF_NONMANIFOLD = 4, MF_NO_BC = 8, MF_BC_NOT_BOUNDARY = 16,
                MF_BC_UNKNOWN = 32, MF_BC_DUP = 64, MF_HASH_FULL = 128 };

static const unsigned long long EMPTY_KEY = ~0ull;

__device__ __forceinline__ unsigned long long edge_key(int a, int b) {
    unsigned lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}
__device__ __forceinline__ unsigned hash_key(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (unsigned)k;
}

__global__ void k_geometry(const double* __restrict__ nodes, const int* __restrict__ elems, int nv, int ne,
                           double* __restrict__ geo, int* flag, unsigned long long* hmax_bits) {
    int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    int v[3];
    bool ok = true;
    for (int i = 0; i < 3; ++i) {
        v[i] = elems[3 * K + i];
        if (v[i] < 0 || v[i] >= nv) ok = false;
    }
    if (!ok) {
        atomicOr(flag, MF_BAD_INDEX);
        return;
    }
    double x0 = nodes[2 * v[0]], y0 = nodes[2 * v[0] + 1];
    double x1 = nodes[2 * v[1]], y1 = nodes[2 * v[1] + 1];
    double x2 = nodes[2 * v[2]], y2 = nodes[2 * v[2] + 1];
    double j00 = x1 - x0, j01 = x2 - x0, j10 = y1 - y0, j11 = y2 - y0;
    double det = j00 * j11 - j01 * j10;
    if (!(det > 0.0)) atomicOr(flag, MF_CLOCKWISE);
    double id = 1.0 / det;
    geo[G_X0 * (size_t)ne + K] = x0;
    geo[G_Y0 * (size_t)ne + K] = y0;
    geo[G_J00 * (size_t)ne + K] = j00;
    geo[G_J01 * (size_t)ne + K] = j01;
    geo[G_J10 * (size_t)ne + K] = j10;
    geo[G_J11 * (size_t)ne + K] = j11;
    geo[G_I00 * (size_t)ne + K] = j11 * id;
    geo[G_I01 * (size_t)ne + K] = -j01 * id;
    geo[G_I10 * (size_t)ne + K] = -j10 * id;
    geo[G_I11 * (size_t)ne + K] = j00 * id;
    geo[G_DET * (size_t)ne + K] = det;
    double l0 = sqrt(j00 * j00 + j10 * j10);
    double l1 = sqrt((x2 - x1) * (x2 - x1) + (y2 - y1) * (y2 - y1));
    double l2 = sqrt(j01 * j01 + j11 * j11);
    double lm = fmax(l0, fmax(l1, l2));
    atomicMax(hmax_bits, (unsigned long long)__double_as_longlong(lm));
}

// Insert every element face into an open-addressing table keyed by its sorted
// vertex pair; the first two owners land in val[2*slot], val[2*slot+1].
__global__ void k_hash_faces(const int* __restrict__ elems, int ne, unsigned long long* keys, int* vals,
                             unsigned mask, int* flag) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * ne) return;
    int K = g / 3, f = g - 3 * K;
    unsigned long long key = edge_key(elems[3 * K + f], elems[3 * K + (f + 1) % 3]);
    unsigned slot = hash_key(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long prev = atomicCAS(&keys[slot], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            if (atomicCAS(&vals[2 * slot], -1, g) != -1)
                if (atomicCAS(&vals[2 * slot + 1], -1, g) != -1) atomicOr(flag, MF_NONMANIFOLD);
            return;
        }
        slot = (slot + 1) & mask;
    }
    atomicOr(flag, MF_HASH_FULL);
}

__device__ __forceinline__ int find_slot(const unsigned long long* keys, unsigned mask, unsigned long long key) {
    unsigned slot = hash_key(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long k = keys[slot];
        if (k == key) return (int)slot;
        if (k == EMPTY_KEY) return -1;
        slot = (slot + 1) & mask;
    }
    return -1;
}

__global__ void k_hash_bc(const int* __restrict__ bc, int nd, int nn, const unsigned long long* keys,
                          int* btype, unsigned mask, int* flag) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nd + nn) return;
    int type = g < nd ? 1 : 2;
    int slot = find_slot(keys, mask, edge_key(bc[2 * g], bc[2 * g + 1]));
    if (slot < 0) {
        atomicOr(flag, MF_BC_UNKNOWN);
        return;
    }
    int prev = atomicCAS(&btype[slot], 0, type);
    if (prev != 0) atomicOr(flag, MF_BC_DUP);
}

__global__ void k_faces(const int* __restrict__ elems, int ne, const unsigned long long* keys, const int* vals,
                        const int* btype, unsigned mask, int* nbr, int* nface, int* ftype, int* bcount, int* flag) {
    int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    int cnt = 0;
    for (int f = 0; f < 3; ++f) {
        int g = 3 * K + f;
        int slot = find_slot(keys, mask, edge_key(elems[g], elems[3 * K + (f + 1) % 3]));
        if (slot < 0) {
            atomicOr(flag, MF_HASH_FULL);
            nbr[f * ne + K] = -1;
            nface[f * ne + K] = -1;
            ftype[f * ne + K] = 0;
            continue;
        }
        int a = vals[2 * slot], b = vals[2 * slot + 1];
        int other = a == g ? b : a;
        if (other >= 0) {
            nbr[f * ne + K] = other / 3;
            nface[f * ne + K] = other % 3;
            ftype[f * ne + K] = 0;
            if (btype[slot] != 0) atomicOr(flag, MF_BC_NOT_BOUNDARY);
        } else {
            nbr[f * ne + K] = -1;
            nface[f * ne + K] = -1;
            int t = btype[slot];
            ftype[f * ne + K] = t;
            if (t == 0) atomicOr(flag, MF_NO_BC);
            ++cnt;
        }
    }
    bcount[K] = cnt;
}

__global__ void k_bidx(const int* __restrict__ ftype, const int* __restrict__ boff, int ne, int* bidx, int* bedge) {
    int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    int o = boff[K];
    for (int f = 0; f < 3; ++f) {
        if (ftype[f * ne + K] != 0) {
            bidx[f * ne + K] = o;
            bedge[o] = 3 * K + f;
            ++o;
        } else {
            bidx[f * ne + K] = -1;
        }
    }
}

// --- exclusive scan of ints (three passes, deterministic) -------------------
#define SCAN_CHUNK 2048
__global__ void k_scan_sums(const int* __restrict__ in, int n, int* bsum) {
    __shared__ double sh[32];
    long base = (long)blockIdx.x * SCAN_CHUNK;
    double s = 0;
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += blockDim.x)
        if (base + i < n) s += in[base + i];
    s = dg_block_sum(s, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = (int)s;
}
// one block: exclusive scan of bsum[nb] in place, total in bsum[nb]
__global__ void k_scan_top(int* bsum, int nb) {
    __shared__ int sh[1024];
    int carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        int tot = sh[1023];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}
__global__ void k_scan_apply(const int* __restrict__ in, int n, const int* __restrict__ bsum, int* out) {
    // 1024 threads x 2 items = SCAN_CHUNK
    __shared__ int sh[1024];
    long base = (long)blockIdx.x * SCAN_CHUNK;
    long i0 = base + 2 * threadIdx.x;
    int a = i0 < n ? in[i0] : 0, b = i0 + 1 < n ? in[i0 + 1] : 0;
    sh[threadIdx.x] = a + b;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int excl = sh[threadIdx.x] - (a + b) + bsum[blockIdx.x];
    if (i0 < n) out[i0] = excl;
    if (i0 + 1 < n) out[i0 + 1] = excl + a;
}

static dg_status exclusive_scan(dg_handle* h, const int* in, int n, int* out, int* bsum, int* total) {
    int nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb == 0) { *total = 0; return DG_OK; }
    k_scan_sums<<<nb, 256, 0, h->stream>>>(in, n, bsum);
    k_scan_top<<<1, 1024, 0, h->stream>>>(bsum, nb);
    k_scan_apply<<<nb, 1024, 0, h->stream>>>(in, n, bsum, out);
    h->nlaunch += 3;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(total, bsum + nb, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

static std::string mesh_flag_text(int f) {
    std::string s;
    if (f & MF_BAD_INDEX) s += " node index out of range;";
    if (f & MF_CLOCKWISE) s += " element not counter-clockwise (or degenerate);";
    if (f & MF_NONMANIFOLD) s += " edge shared by more than two elements;";
    if (f & MF_NO_BC) s += " boundary edge without a boundary condition;";
    if (f & MF_BC_NOT_BOUNDARY) s += " boundary condition on an interior edge;";
    if (f & MF_BC_UNKNOWN) s += " boundary condition on an edge not in the mesh;";
    if (f & MF_BC_DUP) s += " edge listed twice in the boundary conditions;";
    if (f & MF_HASH_FULL) s += " edge table overflow;";
    return "invalid mesh:" + s;
}

extern "C" dg_status dg_mesh_upload(dg_handle* h, const double* nodes, int nv, const int* elems, int ne,
                                    const int* dirichlet, int nd, const int* neumann, int nn) {
    DG_WS_SCOPE(h, DG_WS_MESH);
    if (!h) return DG_ERR_INVALID_ARG;
    if (!nodes || !elems || nv < 3 || ne < 1 || nd < 0 || nn < 0 || (nd > 0 && !dirichlet) ||
        (nn > 0 && !neumann) || ne > (1 << 27))
        return dg_fail(h, DG_ERR_INVALID_ARG, "mesh arrays / sizes");
    DG_CK(h, cudaSetDevice(h->device));
    h->mesh_ok = false;
    h->assembled = false;
    h->bj_ok = false;
    h->ras_ok = false;
    dg_status s;
    if ((s = dg_ensure(h, (void**)&h->nodes, &h->cap_nodes, sizeof(double) * 2 * nv)) != DG_OK) return s;
    if ((s = dg_ensure(h, (void**)&h->elems, &h->cap_elems, sizeof(int) * 3 * (size_t)ne)) != DG_OK) return s;
    if ((s = dg_ensure(h, (void**)&h->geo, &h->cap_geo, sizeof(double) * G_NFIELDS * (size_t)ne)) != DG_OK) return s;
    {
        const size_t fb = sizeof(int) * 3 * (size_t)ne;
        if (h->cap_face < fb) {
            for (int** p : {&h->nbr, &h->nface, &h->ftype, &h->bidx})
                if ((s = dg_realloc(h, (void**)p, fb)) != DG_OK) return s;
            h->cap_face = fb;
        }
    }
    DG_CK(h, cudaMemcpyAsync(h->nodes, nodes, sizeof(double) * 2 * nv, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemcpyAsync(h->elems, elems, sizeof(int) * 3 * (size_t)ne, cudaMemcpyHostToDevice, h->stream));

    // scratch: hash keys, vals, btype, bc list, bcount, boff, bsum, hmax
    unsigned tsize = 1;
    while (tsize < 3u * (unsigned)ne) tsize <<= 1;
    unsigned mask = tsize - 1;
    int nbc = nd + nn;
    int nsb = (ne + SCAN_CHUNK - 1) / SCAN_CHUNK + 1;
    size_t off_keys = 0;
    size_t off_vals = off_keys + sizeof(unsigned long long) * tsize;
    size_t off_bt = off_vals + sizeof(int) * 2 * (size_t)tsize;
    size_t off_bc = off_bt + sizeof(int) * (size_t)tsize;
    size_t off_cnt = off_bc + sizeof(int) * 2 * (size_t)(nbc + 1);
    size_t off_boff = off_cnt + sizeof(int) * (size_t)ne;
    size_t off_bsum = off_boff + sizeof(int) * (size_t)ne;
    size_t off_hm = off_bsum + sizeof(int) * (size_t)nsb + 64;
    off_hm = (off_hm + 15) & ~(size_t)15;
    size_t total = off_hm + 64;
    if ((s = dg_scratch(h, total)) != DG_OK) return s;
    char* sc = (char*)h->scratch;
    unsigned long long* keys = (unsigned long long*)(sc + off_keys);
    int* vals = (int*)(sc + off_vals);
    int* btype = (int*)(sc + off_bt);
    int* bc = (int*)(sc + off_bc);
    int* bcount = (int*)(sc + off_cnt);
    int* boff = (int*)(sc + off_boff);
    int* bsum = (int*)(sc + off_bsum);
    unsigned long long* hm = (unsigned long long*)(sc + off_hm);
    DG_CK(h, cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * tsize, h->stream));
    DG_CK(h, cudaMemsetAsync(vals, 0xff, sizeof(int) * 2 * (size_t)tsize, h->stream));
    DG_CK(h, cudaMemsetAsync(btype, 0, sizeof(int) * (size_t)tsize, h->stream));
    DG_CK(h, cudaMemsetAsync(hm, 0, 8, h->stream));
    DG_CK(h, cudaMemsetAsync(h->dflag, 0, 64, h->stream));
    if (nd) DG_CK(h, cudaMemcpyAsync(bc, dirichlet, sizeof(int) * 2 * nd, cudaMemcpyHostToDevice, h->stream));
    if (nn) DG_CK(h, cudaMemcpyAsync(bc + 2 * nd, neumann, sizeof(int) * 2 * nn, cudaMemcpyHostToDevice, h->stream));

    const int T = 256;
    k_geometry<<<(ne + T - 1) / T, T, 0, h->stream>>>(h->nodes, h->elems, nv, ne, h->geo, h->dflag, hm);
    h->nlaunch += 1;
    int hflag = 0;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaMemcpyAsync(&hflag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (hflag & MF_BAD_INDEX) return dg_fail(h, DG_ERR_MESH, mesh_flag_text(hflag));
    // boundary-condition node ids must be valid too
    for (int i = 0; i < 2 * nd; ++i)
        if (dirichlet[i] < 0 || dirichlet[i] >= nv) return dg_fail(h, DG_ERR_MESH, "Dirichlet node id out of range");
    for (int i = 0; i < 2 * nn; ++i)
        if (neumann[i] < 0 || neumann[i] >= nv) return dg_fail(h, DG_ERR_MESH, "Neumann node id out of range");

    k_hash_faces<<<(3 * ne + T - 1) / T, T, 0, h->stream>>>(h->elems, ne, keys, vals, mask, h->dflag);
    if (nbc) k_hash_bc<<<(nbc + T - 1) / T, T, 0, h->stream>>>(bc, nd, nn, keys, btype, mask, h->dflag);
    k_faces<<<(ne + T - 1) / T, T, 0, h->stream>>>(h->elems, ne, keys, vals, btype, mask, h->nbr, h->nface,
                                                   h->ftype, bcount, h->dflag);
    h->nlaunch += nbc ? 3 : 2;
    DG_LAUNCH_CK(h);
    int nbe = 0;
    if ((s = exclusive_scan(h, bcount, ne, boff, bsum, &nbe)) != DG_OK) return s;
    if ((s = dg_ensure(h, (void**)&h->bedge, &h->cap_bedge, sizeof(int) * (size_t)(nbe > 0 ? nbe : 1))) != DG_OK)
        return s;
    k_bidx<<<(ne + T - 1) / T, T, 0, h->stream>>>(h->ftype, boff, ne, h->bidx, h->bedge);
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    unsigned long long hbits = 0;
    DG_CK(h, cudaMemcpyAsync(&hflag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaMemcpyAsync(&hbits, hm, 8, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (hflag) return dg_fail(h, DG_ERR_MESH, mesh_flag_text(hflag));
    double hmax;
    memcpy(&hmax, &hbits, 8);
    h->nv = nv;
    h->ne = ne;
    h->nbe = nbe;
    h->nint = (3 * ne - nbe) / 2;
    h->ntiles = (ne + DG_TILE - 1) / DG_TILE;
    h->hmax = hmax;
    h->mesh_ok = true;
    return DG_OK;
}

extern "C" dg_status dg_get_info(dg_handle* h, dg_info* out) {
    if (!h || !out) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    int k = h->p.degree;
    memset(out, 0, sizeof(*out));
    out->ne = h->ne;
    out->nv = h->nv;
    out->n_bedges = h->nbe;
    out->n_interior = h->nint;
    out->nb = dg_nb(k);
    out->dofs = (int64_t)h->ne * dg_nb(k);
    out->q_volume = (k + 2) * (k + 2);
    out->q_edge = k + 2;
    out->q_error = (k + 4) * (k + 4);
    for (int i = 0; i < 3; ++i) out->block_bytes[i] = h->assembled ? (int64_t)h->A_bytes[i] : 0;
    return DG_OK;
}

// ---------------------------------------------------------------------------
// point sets
// ---------------------------------------------------------------------------
__global__ void k_points_elem(const double* __restrict__ geo, int ne, const double* __restrict__ r,
                              const double* __restrict__ s, int nq, double* xy) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long)ne * nq) return;
    int K = (int)(g / nq), q = (int)(g - (long)K * nq);
    double x0 = geo[G_X0 * (size_t)ne + K], y0 = geo[G_Y0 * (size_t)ne + K];
    double rr = r[q], ss = s[q];
    xy[2 * g] = x0 + geo[G_J00 * (size_t)ne + K] * rr + geo[G_J01 * (size_t)ne + K] * ss;
    xy[2 * g + 1] = y0 + geo[G_J10 * (size_t)ne + K] * rr + geo[G_J11 * (size_t)ne + K] * ss;
}

// Points of every element face: (K, f, q) at ((K*3 + f)*nq + q), each face run
// from local vertex f to f+1 (counter-clockwise around K).
__global__ void k_points_face(const double* __restrict__ geo, int ne, const double* __restrict__ fr,
                              const double* __restrict__ fs, int nq, double* xy) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long)ne * 3 * nq) return;
    int K = (int)(g / (3 * nq)), fq = (int)(g - (long)K * 3 * nq);
    double rr = fr[fq], ss = fs[fq];
    xy[2 * g] = geo[G_X0 * (size_t)ne + K] + geo[G_J00 * (size_t)ne + K] * rr + geo[G_J01 * (size_t)ne + K] * ss;
    xy[2 * g + 1] = geo[G_Y0 * (size_t)ne + K] + geo[G_J10 * (size_t)ne + K] * rr + geo[G_J11 * (size_t)ne + K] * ss;
}

__global__ void k_points_bdry(const double* __restrict__ geo, int ne, const int* __restrict__ bedge, int nbe,
                              const double* __restrict__ fr, const double* __restrict__ fs, int nq, double* xy,
                              double* normals, int* type, const int* __restrict__ ftype) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long)nbe * nq) return;
    int b = (int)(g / nq), q = (int)(g - (long)b * nq);
    int K = bedge[b] / 3, f = bedge[b] % 3;
    double j00 = geo[G_J00 * (size_t)ne + K], j01 = geo[G_J01 * (size_t)ne + K];
    double j10 = geo[G_J10 * (size_t)ne + K], j11 = geo[G_J11 * (size_t)ne + K];
    double rr = fr[f * nq + q], ss = fs[f * nq + q];
    if (xy) {
        xy[2 * g] = geo[G_X0 * (size_t)ne + K] + j00 * rr + j01 * ss;
        xy[2 * g + 1] = geo[G_Y0 * (size_t)ne + K] + j10 * rr + j11 * ss;
    }
    if (q == 0) {
        // edge vector of face f in physical space: J (V_{f+1} - V_f)
        const double dV[3][2] = {{1, 0}, {-1, 1}, {0, -1}};
        double tx = j00 * dV[f][0] + j01 * dV[f][1], ty = j10 * dV[f][0] + j11 * dV[f][1];
        double len = sqrt(tx * tx + ty * ty);
        if (normals) {
            normals[2 * b] = ty / len;
            normals[2 * b + 1] = -tx / len;
        }
        if (type) type[b] = ftype[f * ne + K];
    }
}

extern "C" dg_status dg_quad_points(dg_handle* h, int which, double* xy) {
    DG_WS_SCOPE(h, DG_WS_MESH);
    if (!h || !xy) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    dg_status s = dg_ensure_tables(h, h->p.degree);
    if (s != DG_OK) return s;
    const TabLayout& L = h->tl;
    const int T = 256;
    if (which == DG_POINTS_VOLUME || which == DG_POINTS_ERROR) {
        int nq = which == DG_POINTS_VOLUME ? L.qk : L.qerr;
        const double* r = h->tab + (which == DG_POINTS_VOLUME ? L.vol_r : L.err_r);
        const double* sv = h->tab + (which == DG_POINTS_VOLUME ? L.vol_s : L.err_s);
        long n = (long)h->ne * nq;
        k_points_elem<<<(unsigned)((n + T - 1) / T), T, 0, h->stream>>>(h->geo, h->ne, r, sv, nq, xy);
    } else if (which == DG_POINTS_BOUNDARY) {
        long n = (long)h->nbe * L.nq;
        if (n > 0)
            k_points_bdry<<<(unsigned)((n + T - 1) / T), T, 0, h->stream>>>(
                h->geo, h->ne, h->bedge, h->nbe, h->tab + L.face_r, h->tab + L.face_s, L.nq, xy, nullptr, nullptr,
                h->ftype);
    } else if (which == DG_POINTS_FACE) {
        long n = (long)h->ne * 3 * L.nq;
        k_points_face<<<(unsigned)((n + T - 1) / T), T, 0, h->stream>>>(h->geo, h->ne, h->tab + L.face_r,
                                                                         h->tab + L.face_s, L.nq, xy);
    } else {
        return dg_fail(h, DG_ERR_INVALID_ARG, "which");
    }
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

extern "C" dg_status dg_boundary_info(dg_handle* h, double* normals, int* type) {
    DG_WS_SCOPE(h, DG_WS_MESH);
    if (!h || (!normals && !type)) return DG_ERR_INVALID_ARG;
    if (!h->mesh_ok) return dg_fail(h, DG_ERR_STATE, "no mesh uploaded");
    dg_status s = dg_ensure_tables(h, h->p.degree);
    if (s != DG_OK) return s;
    const TabLayout& L = h->tl;
    long n = (long)h->nbe * L.nq;
    if (n > 0)
        k_points_bdry<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
            h->geo, h->ne, h->bedge, h->nbe, h->tab + L.face_r, h->tab + L.face_s, L.nq, nullptr, normals, type,
            h->ftype);
    h->nlaunch += n > 0 ? 1 : 0;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

// ---------------------------------------------------------------------------
// copies out of the handle
// ---------------------------------------------------------------------------
extern "C" dg_status dg_get_rhs(dg_handle* h, double* F) {
    if (!h || !F) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    DG_CK(h, cudaMemcpyAsync(F, h->F, sizeof(double) * (size_t)h->ne * dg_nb(h->asm_k), cudaMemcpyDeviceToDevice,
                             h->stream));
    return DG_OK;
}

template <typename T>
__global__ void k_unpack_blocks(const T* __restrict__ A, int ne, int nb, T* out, const int* __restrict__ nbr,
                                int* nbr_out) {
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = 4L * nb * nb;
    if (g >= (long)ne * per) return;
    int K = (int)(g / per);
    int rem = (int)(g - (long)K * per);
    int s = rem / (nb * nb), m = rem - s * nb * nb;
    out[g] = A[dg_blk_index<T>(K, s, m, nb, 4)];
    if (nbr_out && rem < 3) nbr_out[3L * K + rem] = nbr[(size_t)rem * ne + K];
}

extern "C" dg_status dg_get_blocks(dg_handle* h, int dtype, void* out, int* nbr) {
    if (!h || !out) return DG_ERR_INVALID_ARG;
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    int nb = dg_nb(h->asm_k);
    long n = (long)h->ne * 4 * nb * nb;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (dtype == DG_F64 && h->A64)
        k_unpack_blocks<double><<<grid, 256, 0, h->stream>>>(h->A64, h->ne, nb, (double*)out, h->nbr, nbr);
    else if (dtype == DG_F32 && h->A32)
        k_unpack_blocks<float><<<grid, 256, 0, h->stream>>>(h->A32, h->ne, nb, (float*)out, h->nbr, nbr);
    else if (dtype == DG_BF16 && h->A16)
        k_unpack_blocks<__nv_bfloat16><<<grid, 256, 0, h->stream>>>(h->A16, h->ne, nb, (__nv_bfloat16*)out, h->nbr,
                                                                    nbr);
    else
        return dg_fail(h, DG_ERR_STATE, "requested block precision not stored");
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

extern "C" dg_status dg_get_launch_count(dg_handle* h, int64_t* count) {
    if (!h || !count) return DG_ERR_INVALID_ARG;
    *count = h->nlaunch;
    return DG_OK;
}

extern "C" dg_status dg_stream_create(int device, void** stream) {
    if (!stream) return DG_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DG_ERR_CUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreate(&st) != cudaSuccess) return DG_ERR_CUDA;   // blocking w.r.t. the legacy stream
    *stream = (void*)st;
    return DG_OK;
}

extern "C" dg_status dg_stream_destroy(void* stream) {
    if (!stream) return DG_ERR_INVALID_ARG;
    return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
