// dg_nonlin.cu -- the non-linear reaction of Sec. 3 (Eq. (nonlin)):
// alpha u - eps Lap u + b.grad u + r(u) = f with r(u) = c u^p, discretised as
// D v + C v + R v + H(v) = F (Eq. (nonlinsystem)) and solved by Newton's
// method (Eq. (newton)).
//
// H_i(v) = int_K r(u_h) phi_i and HJ_ij(v) = int_K r'(u_h) phi_j phi_i are
// element-local, so HJ adds to the diagonal block (slot 0) of the block-ELL
// operator only.  One warp handles one row i of the 32 elements of a tile
// (lanes are elements, so every reference-table read is a broadcast), with
// the volume rule of the assembly.  The Newton loop runs on the host: per
// step one pass of this kernel over a copy of A (J = A + HJ), the residual,
// and one f64 GMRES solve of J w = -Res with the handle's preconditioner set
// up on J.
#include <math.h>

#include <algorithm>
#include <utility>

#include "dg_kernels.cuh"

// v^p for a small integer p >= 0
__device__ __forceinline__ double dg_ipow(double v, int p) {
    double r = 1.0;
    for (int t = 0; t < p; ++t) r *= v;
    return r;
}

// H [ne*nb] = H(x); with J, J_KK += HJ_K (block-ELL f64, 4 slots); with HJd,
// HJd[K][i][j] = HJ_K(i, j).
template <int NB, int QK>
__global__ void __launch_bounds__(256) k_nonlin(const double* __restrict__ geo, const double* __restrict__ vw,
                                                 const double* __restrict__ vphi, int ne,
                                                 const double* __restrict__ x, int p, double c,
                                                 double* __restrict__ H, double* __restrict__ J,
                                                 double* __restrict__ HJd) {
    const int lane = threadIdx.x & 31;
    const long gw = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ntiles = (ne + 31) >> 5;
    if (gw >= (long)ntiles * NB) return;
    const int tile = (int)(gw / NB);
    const int i = (int)(gw - (long)tile * NB);
    const int K = tile * 32 + lane;
    if (K >= ne) return;
    const double det = __ldg(geo + (size_t)G_DET * ne + K);
    double xk[NB], acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        xk[j] = __ldg(x + (size_t)K * NB + j);
        acc[j] = 0.0;
    }
    double hi = 0.0;
    for (int q = 0; q < QK; ++q) {
        const double* ph = vphi + q * NB;
        double u = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) u = fma(xk[j], __ldg(ph + j), u);
        const double up = dg_ipow(u, p - 1);                  // u^(p-1)
        const double wq = __ldg(vw + q) * det;
        const double pi = __ldg(ph + i);
        hi = fma(wq * c * up * u, pi, hi);                    // r(u) phi_i
        const double t = wq * c * (double)p * up * pi;        // r'(u) phi_i
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = fma(t, __ldg(ph + j), acc[j]);
    }
    H[(size_t)K * NB + i] = hi;
    if (J) {
#pragma unroll
        for (int j = 0; j < NB; ++j) J[dg_blk_index<double>(K, 0, i * NB + j, NB, 4)] += acc[j];
    }
    if (HJd) {
#pragma unroll
        for (int j = 0; j < NB; ++j) HJd[((size_t)K * NB + i) * NB + j] = acc[j];
    }
}

// rhs = F - Ax - H (= -Res); per-block partial sums of rhs^2 and F^2
__global__ void __launch_bounds__(256) k_nl_resid(const double* __restrict__ F, const double* __restrict__ Ax,
                                                   const double* __restrict__ H, double* __restrict__ rhs, long n,
                                                   double* __restrict__ partials) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x) {
        const double f = F[l];
        const double r = f - Ax[l] - H[l];
        rhs[l] = r;
        a = fma(r, r, a);
        b = fma(f, f, b);
    }
    a = dg_block_sum(a, sh);
    b = dg_block_sum(b, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// out[0] = ||rhs||^2, out[1] = ||F||^2 from nblk block partials (one block)
__global__ void __launch_bounds__(256) k_nl_sum(const double* __restrict__ partials, int nblk,
                                                 double* __restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        a += partials[2 * t];
        b += partials[2 * t + 1];
    }
    a = dg_block_sum(a, sh);
    b = dg_block_sum(b, sh);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

__global__ void __launch_bounds__(256) k_nl_axpy(double* __restrict__ x, const double* __restrict__ w, long n) {
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (long)gridDim.x * blockDim.x)
        x[l] += w[l];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static dg_status nonlin_launch(dg_handle* h, int p, double c, const double* x, double* H, double* J, double* HJd) {
    const int k = h->asm_k;
    dg_status s = dg_ensure_tables(h, k);
    if (s != DG_OK) return s;
    const TabLayout& L = h->tl;
    if (L.qk != (k + 2) * (k + 2)) return dg_fail(h, DG_ERR_STATE, "volume rule of the tables");
    const int ntiles = (h->ne + 31) / 32;
    const int nb = dg_nb(k);
    const unsigned grid = (unsigned)(((long)ntiles * nb + 7) / 8);
    const double* vw = h->tab + L.vol_w;
    const double* vphi = h->tab + L.vol_phi;
    switch (k) {
        case 1:
            k_nonlin<3, 9><<<grid, 256, 0, h->stream>>>(h->geo, vw, vphi, h->ne, x, p, c, H, J, HJd);
            break;
        case 2:
            k_nonlin<6, 16><<<grid, 256, 0, h->stream>>>(h->geo, vw, vphi, h->ne, x, p, c, H, J, HJd);
            break;
        case 3:
            k_nonlin<10, 25><<<grid, 256, 0, h->stream>>>(h->geo, vw, vphi, h->ne, x, p, c, H, J, HJd);
            break;
        default:
            return dg_fail(h, DG_ERR_INVALID_ARG, "degree");
    }
    h->nlaunch += 1;
    DG_LAUNCH_CK(h);
    return DG_OK;
}

static dg_status nonlin_checks(dg_handle* h, int p, double c) {
    if (!h->assembled) return dg_fail(h, DG_ERR_STATE, "not assembled");
    if (!h->A64) return dg_fail(h, DG_ERR_STATE, "the f64 blocks are required");
    if (h->b_inst_active) return dg_fail(h, DG_ERR_STATE, "not in batch mode");
    if (p < 1 || p > 4 || !isfinite(c)) return dg_fail(h, DG_ERR_INVALID_ARG, "r(u) = c u^p needs p in 1..4, finite c");
    return DG_OK;
}

extern "C" dg_status dg_nonlinear_global(dg_handle* h, int p, double c, const double* x, double* H, double* HJ) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x || !H) return DG_ERR_INVALID_ARG;
    dg_status s = nonlin_checks(h, p, c);
    if (s != DG_OK) return s;
    DG_CK(h, cudaSetDevice(h->device));
    return nonlin_launch(h, p, c, x, H, nullptr, HJ);
}

// Swaps the f64 operator with the Jacobian for the linear solves and back;
// the preconditioner then belongs to whichever operator was set up last.
struct OperatorSwap {
    dg_handle* h;
    bool on = false;
    void set(bool want) {
        if (want != on) {
            std::swap(h->A64, h->J64);
            h->bj_ok = false;
            h->ras_ok = false;
            on = want;
        }
    }
    ~OperatorSwap() { set(false); }
};

extern "C" dg_status dg_newton_solve(dg_handle* h, int p, double c, int max_newton, double lin_tol, const double* F,
                                     double* x, dg_solve_info* info) {
    DG_WS_SCOPE(h, DG_WS_SOLVER);
    if (!h || !x) return DG_ERR_INVALID_ARG;
    h->basis = nullptr;
    dg_status s = nonlin_checks(h, p, c);
    if (s != DG_OK) return s;
    if (max_newton < 1 || !(lin_tol > 0.0 && lin_tol < 1.0))
        return dg_fail(h, DG_ERR_INVALID_ARG, "max_newton >= 1, 0 < lin_tol < 1");
    if (h->p.precond == DG_PRECOND_MLP)
        return dg_fail(h, DG_ERR_INVALID_ARG, "the Newton steps take block Jacobi, Schwarz or none");
    DG_CK(h, cudaSetDevice(h->device));
    if (!F) F = h->F;
    if (!dg_aligned16(F) || !dg_aligned16(x)) return dg_fail(h, DG_ERR_INVALID_ARG, "F and x must be 16-byte aligned");
    const long n = (long)h->ne * dg_nb(h->asm_k);
    const long ld = (n + 31) / 32 * 32;   // keeps every vector 16-byte aligned
    const int gx = (int)std::min<long>(1024, (n + 255) / 256);
    // rhs, Ax, H, w (ld each), partials [2 gx], sums [2]
    const size_t need = sizeof(double) * (4 * (size_t)ld + 2 * (size_t)gx + 2);
    if ((s = dg_ensure(h, (void**)&h->nl_buf, &h->cap_nl, need)) != DG_OK) return s;
    if ((s = dg_ensure(h, (void**)&h->J64, &h->cap_J64, h->A_bytes[0])) != DG_OK) return s;
    double* rhs = h->nl_buf;
    double* Ax = rhs + ld;
    double* Hv = Ax + ld;
    double* w = Hv + ld;
    double* partials = w + ld;
    double* sums = partials + 2 * gx;
    DG_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));   // v^0 = 0
    const double tol = h->p.tol;
    OperatorSwap swap{h};
    int steps = 0, lin_its = 0;
    double rel = 1.0, hs[2] = {0.0, 0.0};
    bool converged = false;
    for (;;) {
        // J = A + HJ(v), H(v), rhs = F - A v - H(v) = -Res
        DG_CK(h, cudaMemcpyAsync(h->J64, h->A64, h->A_bytes[0], cudaMemcpyDeviceToDevice, h->stream));
        if ((s = nonlin_launch(h, p, c, x, Hv, h->J64, nullptr)) != DG_OK) return s;
        if ((s = dg_launch_apply(h, DG_F64, x, Ax)) != DG_OK) return s;
        k_nl_resid<<<gx, 256, 0, h->stream>>>(F, Ax, Hv, rhs, n, partials);
        k_nl_sum<<<1, 256, 0, h->stream>>>(partials, gx, sums);
        h->nlaunch += 2;
        DG_LAUNCH_CK(h);
        DG_CK(h, cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, h->stream));
        DG_CK(h, cudaStreamSynchronize(h->stream));
        rel = hs[1] > 0.0 ? sqrt(hs[0] / hs[1]) : sqrt(hs[0]);
        if (!isfinite(rel)) return dg_fail(h, DG_ERR_NONFINITE, "NaN/Inf in the Newton residual");
        if (rel <= tol) {
            converged = true;
            break;
        }
        if (steps >= max_newton) break;
        // J w = -Res by restarted GMRES with the preconditioner set up on J
        swap.set(true);
        h->p.tol = lin_tol;
        dg_solve_info li{};
        s = dg_gmres_solve(h, rhs, w, &li);
        h->p.tol = tol;
        swap.set(false);
        if (s != DG_OK && s != DG_NOT_CONVERGED) return s;
        lin_its += li.iterations;
        k_nl_axpy<<<gx, 256, 0, h->stream>>>(x, w, n);
        h->nlaunch += 1;
        DG_LAUNCH_CK(h);
        ++steps;
    }
    if (info) {
        info->iterations = lin_its;
        info->restarts = 0;
        info->outer = steps;
        info->relres = rel;
        info->status = converged ? DG_OK : DG_NOT_CONVERGED;
    }
    h->err.clear();
    if (!converged) return dg_fail(h, DG_NOT_CONVERGED, "Newton did not reach the tolerance");
    return DG_OK;
}
