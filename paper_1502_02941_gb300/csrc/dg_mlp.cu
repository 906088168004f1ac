// dg_mlp.cu -- the learned element-local right preconditioner.
//
// Not part of the paper's method: a small network layered on it.  For element
// K with face neighbours L0..L2 and residual r:
//   s   = sqrt(sum of r^2 over K, L0, L1, L2 / (4 nb)),
//   x   = [r_K, r_L0, r_L1, r_L2] / s  ++  [log10(eps)/6 + 1, b_x, b_y, alpha]
//         (zeros for a missing neighbour; b at the element centroid),
//   y   = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4   (width 128),
//   z_K = A_KK^-1 (r_K + s sigma y_K)      (A_KK^-1: the block-Jacobi inverse).
// Training pairs come from the method's own f64 solves: the residuals
// r = F - A x_k of its iterates, each paired with the one-layer-overlap patch
// correction w (w_K from solving the patch system of K and its face
// neighbours: the restricted additive Schwarz correction).  The network works
// in residual space: its target is t_K = (A_KK w_K - r_K)/s (minus the
// neighbours' coupling terms of the patch solution), so an error in y costs
// the same in the preconditioned residual whatever the conditioning of A_KK;
// sigma = RMS of all targets, and the loss is the mean of |y - t/sigma|^2 / 2,
// minimised by Adam.  The f32 master
// weights are rounded to bf16 for every forward/backward pass, so the trained
// network is the one deployed; training runs as f32 GEMMs on CUDA cores,
// inference as a fused tensor-core kernel (bf16 mma, f32 accumulate) with the
// packed weights resident in shared memory of a persistent grid.
#include <math.h>
#include <string.h>

#include <vector>

#include "dg_kernels.cuh"

#define MW DG_MLP_WIDTH

// ---------------------------------------------------------------------------
// parameter layout
// ---------------------------------------------------------------------------
struct MlpOff {
    long W1, b1, W2, b2, W3, b3, W4, b4, sig, P;
};
static MlpOff mlp_off(int nb) {
    const int din = 4 * nb + DG_MLP_NFEAT;
    MlpOff o;
    long p = 0;
    o.W1 = p; p += (long)MW * din;
    o.b1 = p; p += MW;
    o.W2 = p; p += (long)MW * MW;
    o.b2 = p; p += MW;
    o.W3 = p; p += (long)MW * MW;
    o.b3 = p; p += MW;
    o.W4 = p; p += (long)nb * MW;
    o.b4 = p; p += nb;
    o.sig = p; p += 1;     // fixed output scale sigma (set from the targets at the start of training)
    o.P = p;
    return o;
}

extern "C" dg_status dg_mlp_num_params(int degree, int64_t* n) {
    if (degree < 1 || degree > DG_MAXK || !n) return DG_ERR_INVALID_ARG;
    *n = mlp_off(dg_nb(degree)).P;
    return DG_OK;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16r(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform in [-a, a) from a counter-based hash
__global__ void k_mlp_init(float* theta, long P, MlpOff o, int din, int nb, unsigned long long seed) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
        float bound = 0.f;
        if (i < o.b1) bound = sqrtf(6.f / din);
        else if (i >= o.W2 && i < o.b2) bound = sqrtf(6.f / MW);
        else if (i >= o.W3 && i < o.b3) bound = sqrtf(6.f / MW);
        else if (i >= o.W4 && i < o.b4) bound = 0.1f * sqrtf(3.f / MW);   // small output layer: start near BJ
        const unsigned long long z = mix64(seed ^ (unsigned long long)i * 0x632BE59BD9B4E019ull);
        const float u = (float)((z >> 40) * (1.0 / 16777216.0));   // [0,1)
        theta[i] = i == o.sig ? 1.f : bound * (2.f * u - 1.f);
    }
}

__global__ void k_mlp_round(const float* __restrict__ theta, float* __restrict__ wr, long P) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x)
        wr[i] = i == P - 1 ? theta[i] : bf16r(theta[i]);   // the last entry is the f32 output scale
}

// Adam (bias-corrected); refreshes the bf16-rounded working copy.
__global__ void k_mlp_adam(float* theta, const float* __restrict__ g, float* m, float* v, float* wr, long P, float lr,
                           float c1, float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        theta[i] = th;
        wr[i] = i == P - 1 ? th : bf16r(th);
    }
}

// ---------------------------------------------------------------------------
// f32 tiled GEMM for training:  C[MxN] = op(A)[MxK] op(B)[KxN]  (+ epilogue)
//   TA: A stored [K][M] (op = transpose) else [M][K];  TB: B stored [N][K] else [K][N]
//   epilogue: + bias[n]; relu; * (mask[m][n] > 0)
// ---------------------------------------------------------------------------
#define GT 64
#define GK 16
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                                const float* __restrict__ bias, int relu, const float* __restrict__ mask,
                                                int ldm) {
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int t = threadIdx.x; t < GK * GT; t += 256) {
            const int kk = t / GT, mm = t % GT;
            const int gm = m0 + mm, gk = k0 + kk;
            float a = 0.f;
            if (gm < M && gk < K) a = TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
            As[kk][mm] = a;
            const int gn = n0 + mm;
            float b = 0.f;
            if (gn < N && gk < K) b = TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
            Bs[kk][mm] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) acc[i][jn] = fmaf(a[i], b[jn], acc[i][jn]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + jn;
            if (gm >= M || gn >= N) continue;
            float c = acc[i][jn];
            if (bias) c += bias[gn];
            if (relu) c = fmaxf(c, 0.f);
            if (mask && !(mask[(long)gm * ldm + gn] > 0.f)) c = 0.f;
            C[(long)gm * ldc + gn] = c;
        }
}

template <bool TA, bool TB>
static void sgemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                  int ldc, const float* bias = nullptr, int relu = 0, const float* mask = nullptr, int ldm = 0) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_sgemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, ldm);
}

// column sums of D [rows][n] into out[n]
__global__ void k_colsum(const float* __restrict__ D, int rows, int n, float* __restrict__ out) {
    const int c = blockIdx.x;
    __shared__ double sh[32];
    double s = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s += D[(long)r * n + c];
    s = dg_block_sum(s, sh);
    if (threadIdx.x == 0) out[c] = (float)s;
}

// D = (Y - T) / rows; loss = sum 0.5 (Y - T)^2 / rows
__global__ void k_mlp_lossd(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ D, long cnt,
                            int rows, double* loss) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        D[i] = d / rows;
        a += 0.5 * (double)d * (double)d;
    }
    a = dg_block_sum(a, sh);
    if (threadIdx.x == 0) atomicAdd(loss, a / rows);
}

// gather rows idx of X / T into contiguous batches
__global__ void k_mlp_gather(const float* __restrict__ X, const float* __restrict__ T, int din, int nb, long nrows,
                             int B, unsigned long long seed, int step, float* __restrict__ Xb, float* __restrict__ Tb,
                             const float* __restrict__ sigma) {
    const float inv = 1.f / *sigma;
    for (int r = blockIdx.x; r < B; r += gridDim.x) {
        const unsigned long long z = mix64(seed ^ ((unsigned long long)step << 32) ^ (unsigned long long)r);
        const long src = (long)(z % (unsigned long long)nrows);
        for (int c = threadIdx.x; c < din; c += blockDim.x) Xb[(long)r * din + c] = X[src * din + c];
        for (int c = threadIdx.x; c < nb; c += blockDim.x) Tb[(long)r * nb + c] = T[src * nb + c] * inv;
    }
}

// Loss and gradient of the network (weights wr) on rows Xb/Tb (device).  ws
// holds H1,H2,H3 [B][128], Y/D [B][nb], dH [B][128] x 2.
template <bool TA, bool TB>
static int tcgemm(cudaStream_t s, int nsm, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                  float* C, int ldc, const float* bias, int relu, const float* mask, int ldm, float* part, int* err);

// Where the GEMMs of a training step run: the f32 CUDA-core tiles (k_sgemm) or
// the tensor cores with bf16 operands and f32 accumulation (tcgemm).
struct GemmSel {
    bool tc;
    int nsm;
    float* part;
    int* err;
    int launches;   // kernels launched so far
};
template <bool TA, bool TB>
static void gemm_sel(GemmSel& g, cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* B,
                     int ldb, float* C, int ldc, const float* bias = nullptr, int relu = 0,
                     const float* mask = nullptr, int ldm = 0) {
    if (g.tc) {
        g.launches += tcgemm<TA, TB>(s, g.nsm, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, ldm, g.part, g.err);
    } else {
        sgemm<TA, TB>(s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, ldm);
        ++g.launches;
    }
}

static void mlp_loss_grad(cudaStream_t st, const MlpState& S, const MlpOff& o, const float* Xb, const float* Tb,
                          int B, float* ws, float* grad, double* loss_dev, GemmSel& gs) {
    const int din = S.din, nb = S.nb;
    const float* W = S.wr;
    float* H1 = ws;
    float* H2 = H1 + (long)B * MW;
    float* H3 = H2 + (long)B * MW;
    float* Y = H3 + (long)B * MW;
    float* D = Y + (long)B * 16;
    float* G1 = D + (long)B * 16;
    float* G2 = G1 + (long)B * MW;
    // forward
    gemm_sel<false, true>(gs, st, B, MW, din, Xb, din, W + o.W1, din, H1, MW, W + o.b1, 1);
    gemm_sel<false, true>(gs, st, B, MW, MW, H1, MW, W + o.W2, MW, H2, MW, W + o.b2, 1);
    gemm_sel<false, true>(gs, st, B, MW, MW, H2, MW, W + o.W3, MW, H3, MW, W + o.b3, 1);
    gemm_sel<false, true>(gs, st, B, nb, MW, H3, MW, W + o.W4, MW, Y, nb, W + o.b4, 0);
    k_mlp_lossd<<<64, 256, 0, st>>>(Y, Tb, D, (long)B * nb, B, loss_dev);
    // backward
    gemm_sel<true, false>(gs, st, nb, MW, B, D, nb, H3, MW, grad + o.W4, MW);          // gW4 = D^T H3
    k_colsum<<<nb, 256, 0, st>>>(D, B, nb, grad + o.b4);
    gemm_sel<false, false>(gs, st, B, MW, nb, D, nb, W + o.W4, MW, G1, MW, nullptr, 0, H3, MW);   // dH3
    gemm_sel<true, false>(gs, st, MW, MW, B, G1, MW, H2, MW, grad + o.W3, MW);          // gW3 = dH3^T H2
    k_colsum<<<MW, 256, 0, st>>>(G1, B, MW, grad + o.b3);
    gemm_sel<false, false>(gs, st, B, MW, MW, G1, MW, W + o.W3, MW, G2, MW, nullptr, 0, H2, MW);  // dH2
    gemm_sel<true, false>(gs, st, MW, MW, B, G2, MW, H1, MW, grad + o.W2, MW);          // gW2
    k_colsum<<<MW, 256, 0, st>>>(G2, B, MW, grad + o.b2);
    gemm_sel<false, false>(gs, st, B, MW, MW, G2, MW, W + o.W2, MW, G1, MW, nullptr, 0, H1, MW);  // dH1
    gemm_sel<true, false>(gs, st, MW, din, B, G1, MW, Xb, din, grad + o.W1, din);       // gW1
    k_colsum<<<MW, 256, 0, st>>>(G1, B, MW, grad + o.b1);
}

static size_t mlp_ws_floats(int B) { return (size_t)B * (5 * MW + 32); }

__global__ void k_mlp_rms(const float* __restrict__ T, long cnt, double* acc) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x)
        a += (double)T[i] * (double)T[i];
    a = dg_block_sum(a, sh);
    if (threadIdx.x == 0) atomicAdd(acc, a);
}
__global__ void k_mlp_set_sigma(double* acc, long cnt, float* sig, float* sigr) {
    const float v = (float)sqrt(*acc / (double)cnt);
    *sig = v > 0.f ? v : 1.f;
    *sigr = *sig;
    *acc = 0.0;
}

// ---------------------------------------------------------------------------
// features and training rows
// ---------------------------------------------------------------------------
// coefficient and shape features of element K: eps, bx, by, alpha at the
// centroid, and the Jacobian scaled by 1/sqrt(det J)
__device__ __forceinline__ void elem_coef(int K, int ne, const double* __restrict__ geo, const int* inst,
                                          const double* icoef, const double* scoef, float* out) {
    const double* c = inst ? icoef + (size_t)DG_ICOEF * inst[K] : scoef;
    const double x = geo[G_X0 * (size_t)ne + K] + (geo[G_J00 * (size_t)ne + K] + geo[G_J01 * (size_t)ne + K]) / 3.0;
    const double y = geo[G_Y0 * (size_t)ne + K] + (geo[G_J10 * (size_t)ne + K] + geo[G_J11 * (size_t)ne + K]) / 3.0;
    out[0] = (float)(log10(fmax(c[0], 1e-12)) / 6.0 + 1.0);
    out[1] = (float)(c[2] + c[3] * x + c[4] * y);
    out[2] = (float)(c[5] + c[6] * x + c[7] * y);
    out[3] = (float)c[1];
    const double hs = 1.0 / sqrt(geo[G_DET * (size_t)ne + K]);
    out[4] = (float)(geo[G_J00 * (size_t)ne + K] * hs);
    out[5] = (float)(geo[G_J01 * (size_t)ne + K] * hs);
    out[6] = (float)(geo[G_J10 * (size_t)ne + K] * hs);
    out[7] = (float)(geo[G_J11 * (size_t)ne + K] * hs);
}

struct CoefSrc {
    const double* geo;
    const int* inst;
    const double* icoef;
    double scoef[8];
};

// One training row per element: X = features(r), T = (A_KK w_K - r_K)/s.
template <int NB>
__global__ void k_mlp_rows(const double* __restrict__ r, const double* __restrict__ w, const double* __restrict__ A,
                           const int* __restrict__ nbr, int ne, CoefSrc cs, float* __restrict__ X,
                           float* __restrict__ T) {
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    constexpr int DIN = 4 * NB + DG_MLP_NFEAT;
    double p[4][NB];
    double ss = 0.0;
    for (int sl = 0; sl < 4; ++sl) {
        const int L = sl == 0 ? K : nbr[(size_t)(sl - 1) * ne + K];
        for (int i = 0; i < NB; ++i) {
            p[sl][i] = L >= 0 ? r[(size_t)L * NB + i] : 0.0;
            ss += p[sl][i] * p[sl][i];
        }
    }
    const double s = sqrt(ss / (4 * NB)) + 1e-30;
    float* x = X + (size_t)K * DIN;
    for (int sl = 0; sl < 4; ++sl)
        for (int i = 0; i < NB; ++i) x[sl * NB + i] = (float)(p[sl][i] / s);
    elem_coef(K, ne, cs.geo, cs.inst, cs.icoef, cs.scoef, x + 4 * NB);
    for (int i = 0; i < NB; ++i) {
        double t = -r[(size_t)K * NB + i];
        for (int j = 0; j < NB; ++j) t = fma(A[dg_blk_index<double>(K, 0, i * NB + j, NB, 4)], w[(size_t)K * NB + j], t);
        T[(size_t)K * NB + i] = (float)(t / s);
    }
}

// One-layer-overlap patch solve (the restricted additive Schwarz correction):
// for element K and its face neighbours L_f, solve A_P w = r_P on the patch
// P = {K, L_0, L_1, L_2} (f64 Gaussian elimination with partial pivoting) and
// keep w_K.  A_P couples two neighbours only where they share an edge.
template <int NB>
__global__ void __launch_bounds__(64) k_patch_solve(const double* __restrict__ A, const int* __restrict__ nbr,
                                                     const int* __restrict__ nface, const double* __restrict__ r,
                                                     int ne, double* __restrict__ w) {
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= ne) return;
    constexpr int NP = 4 * NB;
    double M[NP][NP + 1];
    int E[4], cnt = 1;
    int slotK[4];            // slot of K in the row of patch element p (p >= 1)
    E[0] = K;
    for (int f = 0; f < 3; ++f) {
        const int L = nbr[(size_t)f * ne + K];
        if (L >= 0) {
            E[cnt] = L;
            slotK[cnt] = 1 + nface[(size_t)f * ne + K];
            ++cnt;
        }
    }
    const int n = cnt * NB;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b <= n; ++b) M[a][b] = 0.0;
    for (int p = 0; p < cnt; ++p) {
        for (int q = 0; q < cnt; ++q) {
            int slot = -1;
            if (p == q) slot = 0;
            else if (p == 0) {
                for (int f = 0; f < 3; ++f)
                    if (nbr[(size_t)f * ne + K] == E[q]) slot = 1 + f;
            } else if (q == 0) {
                slot = slotK[p];
            } else {
                for (int f = 0; f < 3; ++f)
                    if (nbr[(size_t)f * ne + E[p]] == E[q]) slot = 1 + f;
            }
            if (slot < 0) continue;
            for (int i = 0; i < NB; ++i)
                for (int j = 0; j < NB; ++j)
                    M[p * NB + i][q * NB + j] = A[dg_blk_index<double>(E[p], slot, i * NB + j, NB, 4)];
        }
        for (int i = 0; i < NB; ++i) M[p * NB + i][n] = r[(size_t)E[p] * NB + i];
    }
    bool ok = true;
    for (int c = 0; c < n && ok; ++c) {
        int pv = c;
        for (int a = c + 1; a < n; ++a)
            if (fabs(M[a][c]) > fabs(M[pv][c])) pv = a;
        if (!(fabs(M[pv][c]) > 0.0)) {
            ok = false;
            break;
        }
        if (pv != c)
            for (int b = c; b <= n; ++b) {
                const double t = M[c][b];
                M[c][b] = M[pv][b];
                M[pv][b] = t;
            }
        for (int a = c + 1; a < n; ++a) {
            const double l = M[a][c] / M[c][c];
            if (l != 0.0)
                for (int b = c; b <= n; ++b) M[a][b] -= l * M[c][b];
        }
    }
    double x[NP];
    for (int a = n - 1; a >= 0 && ok; --a) {
        double t = M[a][n];
        for (int b = a + 1; b < n; ++b) t -= M[a][b] * x[b];
        x[a] = t / M[a][a];
    }
    for (int i = 0; i < NB; ++i) w[(size_t)K * NB + i] = ok ? x[i] : 0.0;
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        c[i] = a[i] - b[i];
}

// ---------------------------------------------------------------------------
// packed bf16 inference weights
// ---------------------------------------------------------------------------
struct MlpPack {
    long W1, W2, W3, W4, total;   // offsets in bf16 elements
    int dinp;
};
static MlpPack mlp_pack_layout(int din) {
    MlpPack p;
    p.dinp = (din + 15) / 16 * 16;
    p.W1 = 0;
    p.W2 = p.W1 + (long)MW * p.dinp;
    p.W3 = p.W2 + (long)MW * MW;
    p.W4 = p.W3 + (long)MW * MW;
    p.total = p.W4 + (long)DG_MLP_NOUTP * MW;
    return p;
}

__global__ void k_mlp_pack(const float* __restrict__ theta, MlpOff o, MlpPack pk, int din, int nb,
                           __nv_bfloat16* __restrict__ wbf, float* __restrict__ bias) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < pk.total; i += (long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < pk.W2) {
            const long n = i / pk.dinp, k = i % pk.dinp;
            v = k < din ? theta[o.W1 + n * din + k] : 0.f;
        } else if (i < pk.W3) {
            v = theta[o.W2 + (i - pk.W2)];
        } else if (i < pk.W4) {
            v = theta[o.W3 + (i - pk.W3)];
        } else {
            const long n = (i - pk.W4) / MW, k = (i - pk.W4) % MW;
            v = n < nb ? theta[o.W4 + n * MW + k] : 0.f;
        }
        wbf[i] = __float2bfloat16_rn(v);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * MW + DG_MLP_NOUTP + 1; i += gridDim.x * blockDim.x) {
        float v;
        if (i < MW) v = bf16r(theta[o.b1 + i]);
        else if (i < 2 * MW) v = bf16r(theta[o.b2 + i - MW]);
        else if (i < 3 * MW) v = bf16r(theta[o.b3 + i - 2 * MW]);
        else if (i < 3 * MW + DG_MLP_NOUTP) v = (i - 3 * MW) < nb ? bf16r(theta[o.b4 + i - 3 * MW]) : 0.f;
        else v = theta[o.sig];   // the output scale stays f32
        bias[i] = v;
    }
}

// ---------------------------------------------------------------------------
// fused tensor-core inference (tcgen05: accumulators in tensor memory)
// ---------------------------------------------------------------------------
// CTAs of 128 threads (two per SM where the shared memory fits) walk 128-row
// tiles (row = element).  Thread t
// owns row t: it builds the row's features, and after each layer reads row t
// of the accumulator (TMEM lane t).  Thread 0 issues the tcgen05.mma
// instructions of a layer (M = 128, N = 128 or 16, K = 16 each, bf16 operands
// from shared memory, f32 accumulation in TMEM) and commits them to an
// mbarrier that all threads wait on.  Operands use the K-major layout without
// swizzle: 8-row x 16-byte core matrices, LBO = 128 bytes between the core
// matrices along K, SBO between 8-row groups (K/8 * 128 bytes).
#define MLP_ROWS 128
#define MLP_THREADS 128
#define MLP_ACT_SBO 2048                  // activation tile: 128 columns -> 16 core matrices per 8-row group
#define MLP_WAIT_LIMIT (1u << 26)         // mbarrier polls before the kernel gives up (error flag)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 64-bit shared-memory matrix descriptor: start address, leading and stride
// byte offsets (each >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void smem_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive f32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Wait for phase `parity` of the mbarrier, at most MLP_WAIT_LIMIT polls;
// false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < MLP_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Byte offset of element (row, k) in a K-major core-matrix tile whose 8-row
// groups are sbo bytes apart.
__device__ __forceinline__ uint32_t cm_off(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// 8 f32 values as 8 bf16 (one 16-byte unit of a core matrix row)
__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
    uint4 u;
    u.x = __bfloat16_as_ushort(__float2bfloat16_rn(v[0])) | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[1])) << 16);
    u.y = __bfloat16_as_ushort(__float2bfloat16_rn(v[2])) | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[3])) << 16);
    u.z = __bfloat16_as_ushort(__float2bfloat16_rn(v[4])) | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[5])) << 16);
    u.w = __bfloat16_as_ushort(__float2bfloat16_rn(v[6])) | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[7])) << 16);
    return u;
}

// The coefficient and shape features of elem_coef in f32 (they are rounded to
// bf16 for the network).
__device__ __forceinline__ void elem_coef32(int K, int ne, const double* __restrict__ geo, const int* inst,
                                            const double* icoef, const double* scoef, float* out) {
    const double* c = inst ? icoef + (size_t)DG_ICOEF * inst[K] : scoef;
    const float j00 = (float)geo[G_J00 * (size_t)ne + K], j01 = (float)geo[G_J01 * (size_t)ne + K];
    const float j10 = (float)geo[G_J10 * (size_t)ne + K], j11 = (float)geo[G_J11 * (size_t)ne + K];
    const float x = (float)geo[G_X0 * (size_t)ne + K] + (j00 + j01) * (1.f / 3.f);
    const float y = (float)geo[G_Y0 * (size_t)ne + K] + (j10 + j11) * (1.f / 3.f);
    out[0] = log10f(fmaxf((float)c[0], 1e-12f)) * (1.f / 6.f) + 1.f;
    out[1] = (float)c[2] + (float)c[3] * x + (float)c[4] * y;
    out[2] = (float)c[5] + (float)c[6] * x + (float)c[7] * y;
    out[3] = (float)c[1];
    const float hs = rsqrtf((float)geo[G_DET * (size_t)ne + K]);
    out[4] = j00 * hs;
    out[5] = j01 * hs;
    out[6] = j10 * hs;
    out[7] = j11 * hs;
}

struct MlpRun {
    const __nv_bfloat16* wbf;
    const float* bias;
    MlpPack pk;
    CoefSrc cs;
    const int* on;            // global enable flag (NULL = on)
    const int* iuse;          // per-instance enable flags (batch) or NULL
    const float* B32;         // block-Jacobi inverses A_KK^-1 (f32 copy)
    int* err;                 // device flag: an mbarrier wait ran out
};

// Shared-memory layout of k_mlp_tc (byte offsets, 1024-aligned operand tiles).
struct MlpSmem {
    uint32_t w1, w2, w3, w4, act, bias, s, k, bar, slot, total;
};
__host__ __device__ inline MlpSmem mlp_smem_layout(int dinp) {
    MlpSmem L;
    uint32_t o = 0;
    L.w1 = o; o += (uint32_t)MW * dinp * 2;
    o = (o + 1023u) & ~1023u;
    L.w2 = o; o += MW * MW * 2;
    L.w3 = o; o += MW * MW * 2;
    L.w4 = o; o += DG_MLP_NOUTP * MW * 2;
    o = (o + 1023u) & ~1023u;
    L.act = o; o += MLP_ROWS * MW * 2;
    L.bias = o; o += sizeof(float) * (3 * MW + DG_MLP_NOUTP + 4);
    L.s = o; o += sizeof(float) * MLP_ROWS;
    L.k = o; o += sizeof(int) * MLP_ROWS;
    o = (o + 15u) & ~15u;
    L.bar = o; o += 16;
    L.slot = o; o += 16;
    L.total = o + 1024;   // slack to align the dynamic base to 1024 bytes
    return L;
}

// Copy a row-major [N][K] bf16 matrix into the core-matrix layout (16 bytes
// per thread and step).
__device__ __forceinline__ void stage_cm(const __nv_bfloat16* __restrict__ src, int N, int K, unsigned char* dst) {
    const int units = N * (K / 8);
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        const int n = u / (K / 8), k8 = u - n * (K / 8);
        *reinterpret_cast<uint4*>(dst + cm_off(n, k8 * 8, (uint32_t)K * 16u)) =
            *reinterpret_cast<const uint4*>(src + (size_t)n * K + k8 * 8);
    }
}

// z_K += A_KK^-1 (scale * s_K * sigma * y_K) for every element (r, z vectors of
// type TV, selected through the solver control exactly like the block-Jacobi
// apply); with Xin != NULL: y for precomputed feature rows (parity tests).
template <int NB, typename TV>
__global__ void __launch_bounds__(MLP_THREADS, 2) k_mlp_tc(const TV* __restrict__ r0p, TV* __restrict__ z0p,
                                                            const int* __restrict__ nbr, int ne, MlpRun R, DevCtl ctl,
                                                            VecSel sr, VecSel sz, const float* __restrict__ Xin,
                                                            float* __restrict__ Yout) {
    if (ctl.active && !*ctl.active) return;
    if (R.on && !*R.on) return;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023u) & ~(uintptr_t)1023u);
    constexpr int DIN = 4 * NB + DG_MLP_NFEAT;
    constexpr int DINP = (DIN + 15) / 16 * 16;   // = R.pk.dinp (checked by the launcher)
    const MlpSmem SL = mlp_smem_layout(DINP);
    float* sb = reinterpret_cast<float*>(sm + SL.bias);
    float* ss = reinterpret_cast<float*>(sm + SL.s);
    int* sk = reinterpret_cast<int*>(sm + SL.k);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SL.bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + SL.slot);
    unsigned char* act = sm + SL.act;
    const int t = threadIdx.x, warp = t >> 5;
    // weights (core-matrix layout) and biases once per CTA
    stage_cm(R.wbf + R.pk.W1, MW, DINP, sm + SL.w1);
    stage_cm(R.wbf + R.pk.W2, MW, MW, sm + SL.w2);
    stage_cm(R.wbf + R.pk.W3, MW, MW, sm + SL.w3);
    stage_cm(R.wbf + R.pk.W4, DG_MLP_NOUTP, MW, sm + SL.w4);
    for (int i = t; i < 3 * MW + DG_MLP_NOUTP + 1; i += blockDim.x) sb[i] = R.bias[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(MW)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 TMEM lanes
    const uint32_t s_act = smem_u32(act);
    const uint32_t s_w[4] = {smem_u32(sm + SL.w1), smem_u32(sm + SL.w2), smem_u32(sm + SL.w3), smem_u32(sm + SL.w4)};
    const int kdim[4] = {DINP, MW, MW, MW};
    const TV* __restrict__ r = Xin ? nullptr : sel(r0p, sr);
    TV* __restrict__ z = Xin ? nullptr : sel(z0p, sz);
    const int ntile = (ne + MLP_ROWS - 1) / MLP_ROWS;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        // ---- features of row t (f32), written as bf16 in the core-matrix layout
        {
            const int K = tile * MLP_ROWS + t;
            bool live = K < ne;
            if (live && ctl.inst) live = ctl.iactive[ctl.inst[K]] && (!R.iuse || R.iuse[ctl.inst[K]]);
            float xv[DINP];
#pragma unroll
            for (int c = 0; c < DINP; ++c) xv[c] = 0.f;
            float sc_row = 0.f;
            if (live && Xin) {
                for (int c = 0; c < DIN; ++c) xv[c] = Xin[(size_t)K * DIN + c];
                sc_row = 1.f;
            } else if (live) {
                float sq = 0.f;
#pragma unroll
                for (int sl = 0; sl < 4; ++sl) {
                    const int L = sl == 0 ? K : nbr[(size_t)(sl - 1) * ne + K];
#pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        const float v = L >= 0 ? (float)r[(size_t)L * NB + i] : 0.f;
                        xv[sl * NB + i] = v;
                        sq = fmaf(v, v, sq);
                    }
                }
                const float sd = sqrtf(sq * (1.f / (4 * NB))) + 1e-30f;
                const float inv = 1.f / sd;
#pragma unroll
                for (int c = 0; c < 4 * NB; ++c) xv[c] *= inv;
                elem_coef32(K, ne, R.cs.geo, R.cs.inst, R.cs.icoef, R.cs.scoef, xv + 4 * NB);
                double sc = 1.0;
                if (ctl.inst) sc = ctl.iscale ? ctl.iscale[ctl.inst[K]] : 1.0;
                else if (ctl.scale) sc = ctl.scale[sr.j ? *sr.j + sr.add : 0];
                sc_row = sd * (float)sc;
            }
#pragma unroll
            for (int k8 = 0; k8 < DINP / 8; ++k8)
                *reinterpret_cast<uint4*>(act + cm_off(t, k8 * 8, MLP_ACT_SBO)) = pack8_bf16(xv + k8 * 8);
            ss[t] = sc_row;
            sk[t] = live ? K : -1;
        }
        // ---- four layers; D (TMEM, 128 lanes x 128 f32 columns) is reused
        for (int layer = 0; layer < 4 && ok; ++layer) {
            smem_fence_async();   // this thread's shared-memory writes -> the tensor core's (async) proxy
            tc_fence_before();
            __syncthreads();
            if (t == 0) {
                tc_fence_after();
                const int N = layer == 3 ? DG_MLP_NOUTP : MW;
                const uint32_t idesc = layer == 3 ? tc_idesc(128, DG_MLP_NOUTP) : tc_idesc(128, MW);
                const uint32_t wsbo = (uint32_t)kdim[layer] * 16u;
                for (int ks = 0; ks < kdim[layer] / 16; ++ks)
                    tc_mma(tmem, tc_desc(s_act + ks * 256u, 128u, MLP_ACT_SBO), tc_desc(s_w[layer] + ks * 256u, 128u, wsbo),
                           idesc, ks > 0 ? 1u : 0u);
                tc_commit(bar);
                (void)N;
            }
            // the give-up decision is block-uniform, so every thread takes the same barriers
            if (__syncthreads_or(mbar_wait(bar, phase) ? 0 : 1)) {
                ok = false;
                if (t == 0) {
                    if (R.err) atomicExch(R.err, 1);
                    mbar_wait(bar, phase);   // one more bounded wait for the MMAs in flight
                }
                break;
            }
            phase ^= 1u;
            tc_fence_after();
            if (layer < 3) {
                // bias + relu of row t, written back as the next layer's A operand
                const float* b = sb + layer * MW;
#pragma unroll 1
                for (int c0 = 0; c0 < MW; c0 += 16) {
                    float v[16];
                    tc_ld16(tlane + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + b[c0 + i], 0.f);
                    *reinterpret_cast<uint4*>(act + cm_off(t, c0, MLP_ACT_SBO)) = pack8_bf16(v);
                    *reinterpret_cast<uint4*>(act + cm_off(t, c0 + 8, MLP_ACT_SBO)) = pack8_bf16(v + 8);
                }
            } else {
                // y = D + b4; z_K += A_KK^-1 (s sigma y) in f32, added to z in TV
                float v[16];
                tc_ld16(tlane, v);
                const int K = sk[t];
                const float sig = sb[3 * MW + DG_MLP_NOUTP];
                if (K >= 0) {
                    float u[NB];
#pragma unroll
                    for (int i = 0; i < NB; ++i) u[i] = v[i] + sb[3 * MW + i];
                    if (Yout) {
#pragma unroll
                        for (int i = 0; i < NB; ++i) Yout[(size_t)K * NB + i] = u[i];
                    } else {
                        const float s = ss[t] * sig;
#pragma unroll
                        for (int i = 0; i < NB; ++i) u[i] *= s;
#pragma unroll
                        for (int i = 0; i < NB; ++i) {
                            float a = 0.f;
#pragma unroll
                            for (int j = 0; j < NB; ++j) a = fmaf(R.B32[dg_blk_index<float>(K, 0, i * NB + j, NB, 1)], u[j], a);
                            z[(size_t)K * NB + i] = (TV)((double)z[(size_t)K * NB + i] + (double)a);
                        }
                    }
                }
            }
        }
    }
    // free the tensor memory: every thread's loads have completed (wait::ld)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MW) : "memory");
}

// ---------------------------------------------------------------------------
// tensor-core GEMM for training (tcgen05, accumulators in tensor memory)
// ---------------------------------------------------------------------------
// C[M x N] = op(A)[M x K] op(B)[K x N] with the epilogue of k_sgemm (bias[n],
// relu, mask), N <= 128: op(A)[m][k] = TA ? A[k lda + m] : A[m lda + k] and
// op(B)[k][n] = TB ? B[n ldb + k] : B[k ldb + n], f32 in global memory.  One
// CTA of 128 threads per 128-row tile of C and K split (blockIdx.y) over
// `splits` equal ranges of whole 64-column chunks.  Per chunk the threads
// gather op(A) (128 x 64) and op(B)^T (Np x 64, Np = N rounded up to 16),
// round them to bf16 into the K-major core-matrix layout (as k_mlp_tc), and
// thread 0 issues four tcgen05.mma (M = 128, N = Np, K = 16; f32 accumulation
// in TMEM) and commits them to an mbarrier.  Thread t then reads row t of the
// accumulator: with one split it applies the epilogue and stores C, otherwise
// it stores its split's partial P[split][m][n] for k_tc_gemm_reduce.
#define TCG_KC 64                          // K columns per staged chunk
#define TCG_SBO (TCG_KC / 8 * 128)         // bytes between 8-row groups of a chunk tile
#define TCG_TILE (128 * TCG_KC * 2)        // bytes of one 128-row bf16 chunk tile
#define TCG_SMEM (3 * TCG_TILE + 1024)     // A and B tiles + slack: at most four CTAs per SM (512 TMEM columns)

template <bool T_, bool ROWK>
__device__ __forceinline__ float tcg_elem(const float* __restrict__ X, int ld, int r, int k) {
    // ROWK: element (r, k) at X[r ld + k]; else at X[k ld + r]
    return ROWK ? X[(long)r * ld + k] : X[(long)k * ld + r];
}

// Gather rows [r0, r0 + rows) x chunk columns [k0, k0 + TCG_KC) of an operand
// whose element (r, k) sits at X[r ld + k] (ROWK) or X[k ld + r], as bf16 core
// matrices.  Entries outside R x K are zero.
template <bool ROWK>
__device__ __forceinline__ void tcg_stage(const float* __restrict__ X, int ld, int R, int K, int r0, int k0, int rows,
                                          unsigned char* dst) {
    const int units = rows * (TCG_KC / 8);
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        // ROWK: consecutive threads take consecutive 8-column pieces of a row
        // (contiguous); else consecutive rows of one piece (contiguous along r)
        const int r = ROWK ? u / (TCG_KC / 8) : u % rows;
        const int k8 = ROWK ? u % (TCG_KC / 8) : u / rows;
        float v[8];
        const int gr = r0 + r;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gk = k0 + k8 * 8 + i;
            v[i] = (gr < R && gk < K) ? tcg_elem<false, ROWK>(X, ld, gr, gk) : 0.f;
        }
        *reinterpret_cast<uint4*>(dst + cm_off(r, k8 * 8, TCG_SBO)) = pack8_bf16(v);
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_tc_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                 const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                                 const float* __restrict__ bias, int relu,
                                                 const float* __restrict__ mask, int ldm, int kchunks,
                                                 float* __restrict__ part, int* err) {
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023u) & ~(uintptr_t)1023u);
    unsigned char* sa = sm;
    unsigned char* sbt = sm + TCG_TILE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * TCG_TILE);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + 2 * TCG_TILE + 16);
    const int t = threadIdx.x, warp = t >> 5;
    const int m0 = blockIdx.x * 128;
    const int Np = (N + 15) / 16 * 16;
    const int kbeg = blockIdx.y * kchunks * TCG_KC;
    const int kend = min(K, kbeg + kchunks * TCG_KC);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t idesc = tc_idesc(128, Np);
    uint32_t phase = 0;
    bool ok = true;
    int nchunk = 0;
    for (int k0 = kbeg; k0 < kend && ok; k0 += TCG_KC, ++nchunk) {
        // op(A) row m, col k: A[m lda + k] unless TA; op(B)^T row n, col k: B[n ldb + k] when TB
        tcg_stage<!TA>(A, lda, M, K, m0, k0, 128, sa);
        tcg_stage<TB>(B, ldb, N, K, 0, k0, Np, sbt);
        smem_fence_async();   // the staged tiles -> the tensor core's (async) proxy
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sbt);
#pragma unroll
            for (int ks = 0; ks < TCG_KC / 16; ++ks)
                tc_mma(tmem, tc_desc(a0 + ks * 256u, 128u, TCG_SBO), tc_desc(b0 + ks * 256u, 128u, TCG_SBO), idesc,
                       (nchunk > 0 || ks > 0) ? 1u : 0u);
            tc_commit(bar);
        }
        // the give-up decision is block-uniform, so every thread takes the same barriers
        if (__syncthreads_or(mbar_wait(bar, phase) ? 0 : 1)) {
            ok = false;
            if (t == 0) {
                if (err) atomicExch(err, 1);
                mbar_wait(bar, phase);   // one more bounded wait for the MMAs in flight
            }
        }
        phase ^= 1u;
        tc_fence_after();
    }
    const int m = m0 + t;
    if (ok && nchunk > 0) {
        const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float v[16];
            tc_ld16(tlane + (uint32_t)c0, v);   // every thread of the warp takes part
            if (m >= M) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = c0 + i;
                if (n >= N) break;
                if (gridDim.y > 1) {
                    part[((size_t)blockIdx.y * M + m) * N + n] = v[i];
                } else {
                    float c = v[i];
                    if (bias) c += bias[n];
                    if (relu) c = fmaxf(c, 0.f);
                    if (mask && !(mask[(long)m * ldm + n] > 0.f)) c = 0.f;
                    C[(long)m * ldc + n] = c;
                }
            }
        }
    } else if (!ok || nchunk == 0) {   // an empty split (or a failed wait) contributes zeros
        if (m < M)
            for (int n = 0; n < N; ++n) {
                if (gridDim.y > 1) part[((size_t)blockIdx.y * M + m) * N + n] = 0.f;
                else C[(long)m * ldc + n] = 0.f;
            }
    }
    // free the tensor memory: every thread's loads have completed (wait::ld)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
}

// C = sum of the splits' partials in split order, then the epilogue.
__global__ void k_tc_gemm_reduce(int M, int N, int splits, const float* __restrict__ part, float* __restrict__ C,
                                 int ldc, const float* __restrict__ bias, int relu, const float* __restrict__ mask,
                                 int ldm) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)M * N) return;
    const int m = (int)(e / N), n = (int)(e - (long)m * N);
    float c = 0.f;
    for (int s = 0; s < splits; ++s) c += part[(size_t)s * M * N + e];
    if (bias) c += bias[n];
    if (relu) c = fmaxf(c, 0.f);
    if (mask && !(mask[(long)m * ldm + n] > 0.f)) c = 0.f;
    C[(long)m * ldc + n] = c;
}

#define TCG_MAX_SPLITS 64
#define TCG_PART_FLOATS ((size_t)TCG_MAX_SPLITS * 128 * 128)   // split-K partials of a <= 128 x 128 product

// C = op(A) op(B) (+ epilogue) on the tensor cores, N <= 128 (k_tc_gemm).  K is
// split when there are fewer 128-row tiles than SMs (the weight gradients,
// whose K is the batch of rows), into at most TCG_MAX_SPLITS ranges of whole
// chunks; `part` holds TCG_PART_FLOATS floats.  Returns the kernels launched.
template <bool TA, bool TB>
static int tcgemm(cudaStream_t s, int nsm, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                  float* C, int ldc, const float* bias, int relu, const float* mask, int ldm, float* part, int* err) {
    // (per call: the attribute belongs to the current device)
    cudaFuncSetAttribute(k_tc_gemm<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCG_SMEM);
    const int mt = (M + 127) / 128;
    const int chunks = (K + TCG_KC - 1) / TCG_KC;
    int splits = 1;
    if (mt < nsm && chunks > 1) {
        splits = std::min(chunks, std::max(1, 2 * nsm / mt));
        splits = std::min(splits, (int)(TCG_PART_FLOATS / ((size_t)M * N)));
        splits = std::max(1, std::min(splits, TCG_MAX_SPLITS));
    }
    const int kch = (chunks + splits - 1) / splits;
    splits = (chunks + kch - 1) / kch;
    k_tc_gemm<TA, TB><<<dim3(mt, splits), 128, TCG_SMEM, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, ldm,
                                                               kch, part, err);
    if (splits > 1)
        k_tc_gemm_reduce<<<(unsigned)(((long)M * N + 255) / 256), 256, 0, s>>>(M, N, splits, part, C, ldc, bias, relu,
                                                                               mask, ldm);
    return splits > 1 ? 2 : 1;
}

template <int NB, typename TV>
static dg_status launch_mlp(dg_handle* h, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz, const int* iuse,
                            const float* Xin, float* Yout, int ne) {
    MlpState& S = h->mlp;
    MlpRun R;
    R.wbf = S.wbf;
    R.bias = S.bias;
    R.pk = mlp_pack_layout(S.din);
    R.cs.geo = h->geo;
    R.cs.inst = h->b_inst_active ? h->b_inst : nullptr;
    R.cs.icoef = h->b_inst_active ? h->b_icoef : nullptr;
    for (int t = 0; t < 8; ++t) R.cs.scoef[t] = S.coef[t];
    R.on = Xin ? nullptr : S.on;
    R.iuse = iuse;
    R.B32 = h->Binv32;
    R.err = h->dflag + DG_FLAG_MLP_TIMEOUT;
    if (!Xin && !R.B32) return dg_fail(h, DG_ERR_STATE, "the learned correction needs the block-Jacobi set-up");
    if (R.pk.dinp != (4 * NB + DG_MLP_NFEAT + 15) / 16 * 16) return dg_fail(h, DG_ERR_STATE, "MLP input width");
    const size_t smem = mlp_smem_layout(R.pk.dinp).total;
    // the attribute belongs to a device: set once per (thread, device), every call
    // beyond 64 devices
    static thread_local int configured[64][DG_MAXK + 1][2] = {};
    int dummy = 0;
    int& cfg = h->device >= 0 && h->device < 64
                   ? configured[h->device][dg_nb(1) == NB ? 1 : (dg_nb(2) == NB ? 2 : 3)][sizeof(TV) == 8 ? 1 : 0]
                   : dummy;
    if (!cfg) {
        DG_CK(h, cudaFuncSetAttribute(k_mlp_tc<NB, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cfg = 1;
    }
    // as many CTAs per SM as the shared memory holds (two for P1 / P2, whose
    // weights and activation tile take 112 KB; one for P3): one CTA's feature
    // gathers and epilogues then overlap the other's MMAs
    int sms = 0, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_tc<NB, TV>, MLP_THREADS, smem);
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    const int ntile = (ne + MLP_ROWS - 1) / MLP_ROWS;
    const int grid = ntile < per_sm * sms ? ntile : per_sm * sms;
    k_mlp_tc<NB, TV><<<grid, MLP_THREADS, smem, h->stream>>>(r, z, h->nbr, ne, R, ctl, sr, sz, Xin, Yout);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->stream, &cap);
    if (cap == cudaStreamCaptureStatusNone) h->nlaunch += 1;   // captured launches are counted per graph launch
    return DG_OK;
}

// Entry used by the solvers (dg_gmres.cu / dg_batch.cu): z += MLP correction of r.
template <typename TV>
dg_status dg_mlp_correct(dg_handle* h, const TV* r, TV* z, DevCtl ctl, VecSel sr, VecSel sz, const int* iuse) {
    switch (h->mlp.nb) {
        case 3: return launch_mlp<3, TV>(h, r, z, ctl, sr, sz, iuse, nullptr, nullptr, h->ne);
        case 6: return launch_mlp<6, TV>(h, r, z, ctl, sr, sz, iuse, nullptr, nullptr, h->ne);
        case 10: return launch_mlp<10, TV>(h, r, z, ctl, sr, sz, iuse, nullptr, nullptr, h->ne);
    }
    return dg_fail(h, DG_ERR_STATE, "MLP not initialised for this degree");
}
template dg_status dg_mlp_correct<double>(dg_handle*, const double*, double*, DevCtl, VecSel, VecSel, const int*);
template dg_status dg_mlp_correct<float>(dg_handle*, const float*, float*, DevCtl, VecSel, VecSel, const int*);

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static dg_status mlp_alloc(dg_handle* h, int nb) {
    MlpState& S = h->mlp;
    if (S.nb == nb && S.theta) return DG_OK;
    const MlpOff o = mlp_off(nb);
    S.nb = nb;
    S.din = 4 * nb + DG_MLP_NFEAT;
    S.dinp = (S.din + 15) / 16 * 16;
    S.P = o.P;
    dg_status s;
    for (float** p : {&S.theta, &S.wr, &S.m, &S.v, &S.grad})
        if ((s = dg_realloc(h, (void**)p, sizeof(float) * o.P)) != DG_OK) return s;
    const MlpPack pk = mlp_pack_layout(S.din);
    if ((s = dg_realloc(h, (void**)&S.wbf, sizeof(__nv_bfloat16) * pk.total)) != DG_OK) return s;
    if ((s = dg_realloc(h, (void**)&S.bias, sizeof(float) * (3 * MW + DG_MLP_NOUTP + 1))) != DG_OK) return s;
    DG_CK(h, cudaMemsetAsync(S.grad, 0, sizeof(float) * o.P, h->stream));   // the scale entry keeps a zero gradient
    if (!S.on) {
        if ((s = dg_realloc(h, (void**)&S.on, sizeof(int))) != DG_OK) return s;
    }
    S.ready = false;
    S.packed = false;
    S.step = 0;
    S.rows = 0;
    return DG_OK;
}

static dg_status mlp_refresh(dg_handle* h) {
    MlpState& S = h->mlp;
    const MlpOff o = mlp_off(S.nb);
    k_mlp_round<<<256, 256, 0, h->stream>>>(S.theta, S.wr, S.P);
    const MlpPack pk = mlp_pack_layout(S.din);
    k_mlp_pack<<<256, 256, 0, h->stream>>>(S.theta, o, pk, S.din, S.nb, S.wbf, S.bias);
    const int one = 1;
    DG_CK(h, cudaMemcpyAsync(S.on, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaStreamSynchronize(h->stream));
    S.ready = true;
    S.packed = true;
    return DG_OK;
}

extern "C" dg_status dg_mlp_init(dg_handle* h, uint64_t seed) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h) return DG_ERR_INVALID_ARG;
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->p.degree);
    dg_status s = mlp_alloc(h, nb);
    if (s != DG_OK) return s;
    MlpState& S = h->mlp;
    const MlpOff o = mlp_off(nb);
    k_mlp_init<<<256, 256, 0, h->stream>>>(S.theta, S.P, o, S.din, nb, (unsigned long long)seed);
    DG_CK(h, cudaMemsetAsync(S.m, 0, sizeof(float) * S.P, h->stream));
    DG_CK(h, cudaMemsetAsync(S.v, 0, sizeof(float) * S.P, h->stream));
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    S.step = 0;
    return mlp_refresh(h);
}

extern "C" dg_status dg_mlp_set_weights(dg_handle* h, const float* theta, int64_t n) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || !theta) return DG_ERR_INVALID_ARG;
    DG_CK(h, cudaSetDevice(h->device));
    const int nb = dg_nb(h->p.degree);
    dg_status s = mlp_alloc(h, nb);
    if (s != DG_OK) return s;
    if (n != h->mlp.P) return dg_fail(h, DG_ERR_INVALID_ARG, "parameter count does not match the degree");
    DG_CK(h, cudaMemcpyAsync(h->mlp.theta, theta, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    DG_CK(h, cudaMemsetAsync(h->mlp.m, 0, sizeof(float) * n, h->stream));
    DG_CK(h, cudaMemsetAsync(h->mlp.v, 0, sizeof(float) * n, h->stream));
    h->mlp.step = 0;
    return mlp_refresh(h);
}

extern "C" dg_status dg_mlp_get_weights(dg_handle* h, float* theta, int64_t n) {
    if (!h || !theta) return DG_ERR_INVALID_ARG;
    if (!h->mlp.ready) return dg_fail(h, DG_ERR_STATE, "MLP not initialised");
    if (n != h->mlp.P) return dg_fail(h, DG_ERR_INVALID_ARG, "parameter count");
    DG_CK(h, cudaMemcpyAsync(theta, h->mlp.theta, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

extern "C" dg_status dg_mlp_clear_data(dg_handle* h) {
    if (!h) return DG_ERR_INVALID_ARG;
    h->mlp.rows = 0;
    return DG_OK;
}

static dg_status mlp_check_collect(dg_handle* h) {
    if (!h->assembled || !h->A64) return dg_fail(h, DG_ERR_STATE, "assemble with f64 blocks first");
    MlpState& S = h->mlp;
    if (!S.ready || S.nb != dg_nb(h->asm_k)) return dg_fail(h, DG_ERR_STATE, "dg_mlp_init first (same degree)");
    DG_CK(h, cudaSetDevice(h->device));
    return DG_OK;
}

// Append one row per element for the residual r (device f64, unnormalised):
// w = patch-solve correction of r into the scratch vector e, then the rows.
static dg_status mlp_rows_from(dg_handle* h, const double* r, double* e) {
    MlpState& S = h->mlp;
    const int nb = S.nb;
    const long need = S.rows + h->ne;
    if (need > S.cap) {
        long cap = S.cap ? S.cap : 65536;
        while (cap < need) cap *= 2;
        float *X = nullptr, *T = nullptr;
        dg_status s = dg_dev_alloc(h, (void**)&X, sizeof(float) * cap * S.din);
        if (s != DG_OK) return s;
        if ((s = dg_dev_alloc(h, (void**)&T, sizeof(float) * cap * nb)) != DG_OK) {
            dg_dev_free(h, X);
            return s;
        }
        if (S.rows) {
            DG_CK(h, cudaMemcpyAsync(X, S.X, sizeof(float) * S.rows * S.din, cudaMemcpyDeviceToDevice, h->stream));
            DG_CK(h, cudaMemcpyAsync(T, S.T, sizeof(float) * S.rows * nb, cudaMemcpyDeviceToDevice, h->stream));
        }
        DG_CK(h, cudaStreamSynchronize(h->stream));
        dg_dev_free(h, S.X);
        dg_dev_free(h, S.T);
        S.X = X;
        S.T = T;
        S.cap = cap;
    }
    const unsigned gp = (unsigned)((h->ne + 63) / 64);
    switch (nb) {
        case 3: k_patch_solve<3><<<gp, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, r, h->ne, e); break;
        case 6: k_patch_solve<6><<<gp, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, r, h->ne, e); break;
        case 10: k_patch_solve<10><<<gp, 64, 0, h->stream>>>(h->A64, h->nbr, h->nface, r, h->ne, e); break;
    }
    CoefSrc cs;
    cs.geo = h->geo;
    cs.inst = h->b_inst_active ? h->b_inst : nullptr;
    cs.icoef = h->b_inst_active ? h->b_icoef : nullptr;
    for (int t = 0; t < 8; ++t) cs.scoef[t] = S.coef[t];
    float* X = S.X + S.rows * S.din;
    float* T = S.T + S.rows * nb;
    const unsigned grid = (unsigned)((h->ne + 127) / 128);
    switch (nb) {
        case 3: k_mlp_rows<3><<<grid, 128, 0, h->stream>>>(r, e, h->A64, h->nbr, h->ne, cs, X, T); break;
        case 6: k_mlp_rows<6><<<grid, 128, 0, h->stream>>>(r, e, h->A64, h->nbr, h->ne, cs, X, T); break;
        case 10: k_mlp_rows<10><<<grid, 128, 0, h->stream>>>(r, e, h->A64, h->nbr, h->ne, cs, X, T); break;
    }
    h->nlaunch += 2;
    DG_LAUNCH_CK(h);
    S.rows += h->ne;
    return DG_OK;
}

extern "C" dg_status dg_mlp_collect(dg_handle* h, const double* F, const double* xk) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || !xk) return DG_ERR_INVALID_ARG;
    dg_status s = mlp_check_collect(h);
    if (s != DG_OK) return s;
    if (!F) F = h->F;
    const long n = (long)h->ne * h->mlp.nb;
    if ((s = dg_scratch(h, sizeof(double) * 2 * n)) != DG_OK) return s;
    double* r = h->scratch;
    double* e = r + n;
    // r = F - A xk (A xk staged in e)
    if ((s = dg_launch_apply(h, DG_F64, xk, e)) != DG_OK) return s;
    k_sub<<<512, 256, 0, h->stream>>>(F, e, r, n);
    h->nlaunch += 1;
    if ((s = mlp_rows_from(h, r, e)) != DG_OK) return s;
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

extern "C" dg_status dg_mlp_collect_basis(dg_handle* h, int nvec) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || nvec < 1) return DG_ERR_INVALID_ARG;
    dg_status s = mlp_check_collect(h);
    if (s != DG_OK) return s;
    if (!h->basis) return dg_fail(h, DG_ERR_STATE, "no Krylov basis: run an f64 solve first");
    if (nvec > h->basis_n) return dg_fail(h, DG_ERR_INVALID_ARG, "nvec exceeds the basis size (gmres_m + 1)");
    const long n = (long)h->ne * h->mlp.nb;
    if ((s = dg_scratch(h, sizeof(double) * n)) != DG_OK) return s;
    for (int j = 0; j < nvec; ++j)
        if ((s = mlp_rows_from(h, h->basis + (size_t)j * h->basis_ld, h->scratch)) != DG_OK) return s;
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

extern "C" dg_status dg_mlp_num_rows(dg_handle* h, int64_t* rows) {
    if (!h || !rows) return DG_ERR_INVALID_ARG;
    *rows = h->mlp.rows;
    return DG_OK;
}

// Training workspace: activations and gradients of B rows, a batch of rows,
// the loss accumulator, and the split-K partials of the tensor-core GEMMs.
static size_t mlp_ws_part_offset(const MlpState& S, int B) {
    const size_t f = mlp_ws_floats(B) + (size_t)B * (S.din + S.nb) + 2 * sizeof(double) / sizeof(float) + 8;
    return (f + 63) / 64 * 64;   // floats, 256-byte aligned
}
static dg_status mlp_ws(dg_handle* h, int B) {
    MlpState& S = h->mlp;
    const size_t need = sizeof(float) * (mlp_ws_part_offset(S, B) + TCG_PART_FLOATS);
    if (S.ws_cap >= need) return DG_OK;
    dg_status s = dg_realloc(h, (void**)&S.ws, need);
    S.ws_cap = s == DG_OK ? need : 0;
    return s;
}

extern "C" dg_status dg_mlp_train(dg_handle* h, int steps, int batch_rows, float lr, uint64_t seed, float* loss) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || steps < 1 || batch_rows < 1 || !(lr > 0.f)) return DG_ERR_INVALID_ARG;
    MlpState& S = h->mlp;
    if (!S.ready) return dg_fail(h, DG_ERR_STATE, "dg_mlp_init first");
    if (S.rows < 1) return dg_fail(h, DG_ERR_STATE, "no training rows (dg_mlp_collect)");
    DG_CK(h, cudaSetDevice(h->device));
    dg_status s = mlp_ws(h, batch_rows);
    if (s != DG_OK) return s;
    const MlpOff o = mlp_off(S.nb);
    float* ws = S.ws;
    float* Xb = ws + mlp_ws_floats(batch_rows);
    float* Tb = Xb + (size_t)batch_rows * S.din;
    double* lossd = reinterpret_cast<double*>(Tb + (size_t)batch_rows * S.nb + 2);
    lossd = reinterpret_cast<double*>(((uintptr_t)lossd + 7) & ~(uintptr_t)7);
    std::vector<double> hl(steps);
    DG_CK(h, cudaMemsetAsync(lossd, 0, sizeof(double), h->stream));
    if (S.step == 0) {
        // output scale sigma = RMS of the collected targets (kept fixed afterwards)
        k_mlp_rms<<<256, 256, 0, h->stream>>>(S.T, S.rows * S.nb, lossd);
        k_mlp_set_sigma<<<1, 1, 0, h->stream>>>(lossd, S.rows * S.nb, S.theta + o.sig, S.wr + o.sig);
        h->nlaunch += 2;
    }
    // the GEMMs of training on the tensor cores
    GemmSel gs{true, h->nsm, ws + mlp_ws_part_offset(S, batch_rows), h->dflag + DG_FLAG_MLP_TIMEOUT, 0};
    for (int it = 0; it < steps; ++it) {
        k_mlp_gather<<<256, 64, 0, h->stream>>>(S.X, S.T, S.din, S.nb, S.rows, batch_rows, seed, S.step + it, Xb, Tb,
                                                S.theta + o.sig);
        DG_CK(h, cudaMemsetAsync(lossd, 0, sizeof(double), h->stream));
        mlp_loss_grad(h->stream, S, o, Xb, Tb, batch_rows, ws, S.grad, lossd, gs);
        ++S.step;
        const float c1 = 1.f - powf(0.9f, (float)S.step), c2 = 1.f - powf(0.999f, (float)S.step);
        k_mlp_adam<<<512, 256, 0, h->stream>>>(S.theta, S.grad, S.m, S.v, S.wr, S.P, lr, c1, c2);
        h->nlaunch += 7;   // gather, loss, four column sums, Adam
        if (loss) DG_CK(h, cudaMemcpyAsync(&hl[it], lossd, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    DG_LAUNCH_CK(h);
    DG_CK(h, cudaStreamSynchronize(h->stream));
    h->nlaunch += gs.launches;
    if (loss)
        for (int it = 0; it < steps; ++it) loss[it] = (float)hl[it];
    if ((s = dg_mlp_check_timeout(h)) != DG_OK) return s;
    return mlp_refresh(h);
}

// Loss and gradient at the current weights on caller rows (device X [rows][din],
// T [rows][nb] f32); host outputs.
extern "C" dg_status dg_mlp_loss_grad(dg_handle* h, const float* X, const float* T, int rows, double* loss,
                                      float* grad) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || !X || !T || rows < 1) return DG_ERR_INVALID_ARG;
    MlpState& S = h->mlp;
    if (!S.ready) return dg_fail(h, DG_ERR_STATE, "dg_mlp_init first");
    DG_CK(h, cudaSetDevice(h->device));
    dg_status s = mlp_ws(h, rows);
    if (s != DG_OK) return s;
    const MlpOff o = mlp_off(S.nb);
    float* ws = S.ws;
    double* lossd = reinterpret_cast<double*>(((uintptr_t)(ws + mlp_ws_floats(rows) + (size_t)rows * (S.din + S.nb)) + 7) &
                                              ~(uintptr_t)7);
    DG_CK(h, cudaMemsetAsync(lossd, 0, sizeof(double), h->stream));
    GemmSel gs{h->mlp_grad_tc, h->nsm, ws + mlp_ws_part_offset(S, rows), h->dflag + DG_FLAG_MLP_TIMEOUT, 0};
    mlp_loss_grad(h->stream, S, o, X, T, rows, ws, S.grad, lossd, gs);
    h->nlaunch += 5 + gs.launches;   // + the loss and four column sums
    DG_LAUNCH_CK(h);
    if (loss) DG_CK(h, cudaMemcpyAsync(loss, lossd, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (grad) DG_CK(h, cudaMemcpyAsync(grad, S.grad, sizeof(float) * S.P, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return h->mlp_grad_tc ? dg_mlp_check_timeout(h) : DG_OK;
}

// Tensor-core forward on caller feature rows: Y [rows][nb] (device f32).
extern "C" dg_status dg_mlp_forward(dg_handle* h, const float* X, int rows, float* Y) {
    DG_WS_SCOPE(h, DG_WS_LEARNED);
    if (!h || !X || !Y || rows < 1) return DG_ERR_INVALID_ARG;
    MlpState& S = h->mlp;
    if (!S.packed) return dg_fail(h, DG_ERR_STATE, "dg_mlp_init first");
    DG_CK(h, cudaSetDevice(h->device));
    dg_status s;
    switch (S.nb) {
        case 3: s = launch_mlp<3, float>(h, nullptr, nullptr, dctl_none(), vsel_fixed(), vsel_fixed(), nullptr, X, Y, rows); break;
        case 6: s = launch_mlp<6, float>(h, nullptr, nullptr, dctl_none(), vsel_fixed(), vsel_fixed(), nullptr, X, Y, rows); break;
        case 10: s = launch_mlp<10, float>(h, nullptr, nullptr, dctl_none(), vsel_fixed(), vsel_fixed(), nullptr, X, Y, rows); break;
        default: return dg_fail(h, DG_ERR_STATE, "degree");
    }
    if (s != DG_OK) return s;
    DG_LAUNCH_CK(h);
    return dg_mlp_check_timeout(h);
}

// The inference kernel's bounded waits: DG_ERR_TIMEOUT (and the flag cleared)
// if a launch since the last check gave up waiting for its MMAs.  Synchronises.
dg_status dg_mlp_check_timeout(dg_handle* h) {
    int f = 0;
    DG_CK(h, cudaMemcpyAsync(&f, h->dflag + DG_FLAG_MLP_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    if (!f) return DG_OK;
    DG_CK(h, cudaMemsetAsync(h->dflag + DG_FLAG_MLP_TIMEOUT, 0, sizeof(int), h->stream));
    return dg_fail(h, DG_ERR_TIMEOUT, "the learned preconditioner's tensor-core kernel gave up waiting for its MMAs");
}

// Copy collected rows to the host (first `max_rows`).
extern "C" dg_status dg_mlp_get_rows(dg_handle* h, float* X, float* T, int64_t max_rows) {
    if (!h || max_rows < 0) return DG_ERR_INVALID_ARG;
    MlpState& S = h->mlp;
    const long n = max_rows < S.rows ? max_rows : S.rows;
    if (X && n) DG_CK(h, cudaMemcpyAsync(X, S.X, sizeof(float) * n * S.din, cudaMemcpyDeviceToHost, h->stream));
    if (T && n) DG_CK(h, cudaMemcpyAsync(T, S.T, sizeof(float) * n * S.nb, cudaMemcpyDeviceToHost, h->stream));
    DG_CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}
