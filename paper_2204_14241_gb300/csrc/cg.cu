// Conjugate gradient on A = D D^dagger (Eq. linsys), optionally preconditioned with
// P = (K K^dagger)^{-1} (Eq. precon), for k right-hand sides at once.
//
// Precision: HMC_SOLVER_FP64 iterates in complex128. HMC_SOLVER_MIXED iterates in complex64
// and keeps the solution and the true residual in complex128 ("reliable updates": whenever
// the iterated residual has dropped by a factor 1000 since the last update, or meets the
// tolerance, the partial solution is folded into the FP64 solution, the residual is
// recomputed in FP64 as b - A x, and the iteration continues from it with the same search
// direction). Both modes stop on the FP64 true residual ||b - A x|| <= tol ||b||.
//
// Scalars (alpha, beta, norms, flags) live on the device; kernels of right-hand sides that
// have converged return at once. The host looks at the flags every few iterations.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace hmc {

template <typename R> using V16 = std::conditional_t<sizeof(R) == 4, float4, double2>;

__device__ __forceinline__ float4 v_axpy(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 v_axpy(double a, double2 x, double2 y) {
    return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ double v_dot(float4 a, float4 b) {
    return (double)(a.x * b.x + a.y * b.y) + (double)(a.z * b.z + a.w * b.w);
}
__device__ __forceinline__ double v_dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

constexpr int kRedBlocks = 512;   // partial sums per right-hand side for vector reductions

// part[k * gridDim.x + b] = partial Re<a_k, b_k> over the 16-byte units of rhs k
template <typename R>
__global__ void __launch_bounds__(256) k_dot(const V16<R>* __restrict__ a, const V16<R>* __restrict__ b,
                                             int64_t n16, double* __restrict__ part,
                                             const CgScalars* __restrict__ cgs) {
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (cgs && !cgs[k].active) return;
    const V16<R>* ak = a + k * n16;
    const V16<R>* bk = b + k * n16;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        s += v_dot(ak[i], bk[i]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

// x += alpha p; r -= alpha q; partial ||r||^2
template <typename R>
__global__ void __launch_bounds__(256) k_cg_xr(V16<R>* __restrict__ x, V16<R>* __restrict__ r,
                                               const V16<R>* __restrict__ p, const V16<R>* __restrict__ q,
                                               int64_t n16, double* __restrict__ part,
                                               const CgScalars* __restrict__ cgs) {
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (!cgs[k].active) return;
    const R alpha = (R)cgs[k].alpha;
    const int64_t off = k * n16;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        x[off + i] = v_axpy(alpha, p[off + i], x[off + i]);
        const V16<R> rn = v_axpy(-alpha, q[off + i], r[off + i]);
        r[off + i] = rn;
        s += v_dot(rn, rn);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

// Fused complex64 update of plain CG: r -= alpha q; p = r + beta p (beta known before r: see
// k_cg_ab); partial ||r||^2; and x += alpha p every other iteration. An iteration with
// defer set (and beta > 0) leaves x alone and k_cg_beta records carry = alpha / beta; the next one
// adds both terms, recovering the previous direction from the vectors it reads anyway:
// p_prev = (p - r) / beta_prev, so x += alpha p + carry (p - r). One pass over r, p, q, and over x
// on the iterations that update it.
__device__ __forceinline__ float4 v_sub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__global__ void __launch_bounds__(256) k_cg_xrp(float4* __restrict__ x, float4* __restrict__ r, float4* __restrict__ p,
                                                const float4* __restrict__ q, int64_t n16, double* __restrict__ part,
                                                const CgScalars* __restrict__ cgs, int defer) {
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (!cgs[k].active) return;
    const float alpha = (float)cgs[k].alpha, beta = (float)cgs[k].beta, carry = (float)cgs[k].carry;
    const bool skip_x = defer && cgs[k].beta > 0.0;
    const int64_t off = k * n16;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 pv = p[off + i], rv = r[off + i];
        if (!skip_x) x[off + i] = v_axpy(carry, v_sub(pv, rv), v_axpy(alpha, pv, x[off + i]));
        const float4 rn = v_axpy(-alpha, q[off + i], rv);
        r[off + i] = rn;
        p[off + i] = v_axpy(beta, pv, rn);
        s += v_dot(rn, rn);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

__device__ __forceinline__ double row_sum(const double* part, int nblk, double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
    return block_sum(s, red);
}

// alpha = <r, z> / <p, A p>; one block per right-hand side
__global__ void k_cg_alpha(CgScalars* cgs, const double* __restrict__ part, int nblk) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    if (!cgs[k].active) return;
    const double pAp = row_sum(part + (int64_t)k * nblk, nblk, red);
    if (threadIdx.x == 0) {
        cgs[k].pAp = pAp;
        cgs[k].alpha = (pAp > 0.0 && isfinite(pAp)) ? cgs[k].rr / pAp : 0.0;
        if (!isfinite(pAp)) cgs[k].nonfinite = 1;
    }
}

// Plain CG with beta ahead of the residual update: alpha = <r, r> / <p, A p> and
//   ||r - alpha A p||^2 = ||r||^2 - 2 alpha Re<r, A p> + alpha^2 ||A p||^2 = alpha^2 ||A p||^2 - ||r||^2,
// since <r, A p> = <p, A p> for a direction p = r + beta' p' conjugate to the previous one
// (<p', A p> = 0) and alpha <p, A p> = ||r||^2. beta = that norm / ||r||^2 (0 if rounding makes it
// negative, which restarts the direction). The residual norm itself comes from the update pass.
__global__ void k_cg_ab(CgScalars* cgs, const double* __restrict__ part_pap, const double* __restrict__ part_qq,
                        int nblk) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    if (!cgs[k].active) return;
    const double pAp = row_sum(part_pap + (int64_t)k * nblk, nblk, red);
    const double qq = row_sum(part_qq + (int64_t)k * nblk, nblk, red);
    if (threadIdx.x == 0) {
        CgScalars& c = cgs[k];
        c.pAp = pAp;
        const double alpha = (pAp > 0.0 && isfinite(pAp)) ? c.rr / pAp : 0.0;
        const double rnext = alpha * alpha * qq - c.rr;
        c.alpha = alpha;
        c.beta = (c.rr > 0.0 && rnext > 0.0) ? rnext / c.rr : 0.0;
        if (!isfinite(pAp) || !isfinite(qq)) c.nonfinite = 1;
    }
}

// r2 = ||r||^2, rz_new = <r, z> (= r2 without preconditioner), beta (unless set_beta is 0: the
// fused plain update took it from k_cg_ab, and defer says whether that update left x for the next
// iteration, see k_cg_xrp), convergence flags
__global__ void k_cg_beta(CgScalars* cgs, const double* __restrict__ part_r2,
                          const double* __restrict__ part_rz, int nblk, int nblk_rz, double tol2, double delta2,
                          int mixed, int set_beta, int defer) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    if (!cgs[k].active) return;
    const double r2 = row_sum(part_r2 + (int64_t)k * nblk, nblk, red);
    const double rz = part_rz ? row_sum(part_rz + (int64_t)k * nblk_rz, nblk_rz, red) : r2;
    if (threadIdx.x == 0) {
        CgScalars& c = cgs[k];
        if (set_beta) c.beta = c.rr > 0.0 ? rz / c.rr : 0.0;
        else c.carry = (defer && c.beta > 0.0) ? c.alpha / c.beta : 0.0;
        c.rr = rz;
        c.r2 = r2;
        c.iters += 1;
        if (!isfinite(r2) || !isfinite(rz)) c.nonfinite = 1;
        if (r2 <= tol2 * c.b2 || (mixed && r2 < delta2 * c.r2_max)) c.need_ru = 1;
    }
}

// Initial scalars: b2 = ||b||^2 from part_b2; r2 = r2_max = ||b - A x0||^2 from part_r2 (or
// b2 for a zero start). A right-hand side is active unless b = 0 or x0 already meets tol.
__global__ void k_cg_start(CgScalars* cgs, const double* __restrict__ part_b2, int nblk_b2,
                           const double* __restrict__ part_r2, int nblk_r2, double tol2) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    const double b2 = row_sum(part_b2 + (int64_t)k * nblk_b2, nblk_b2, red);
    const double r2 = part_r2 ? row_sum(part_r2 + (int64_t)k * nblk_r2, nblk_r2, red) : b2;
    if (threadIdx.x == 0) {
        CgScalars c = {};
        c.b2 = b2;
        c.r2 = r2;
        c.r2_max = r2;
        c.r2true = r2;
        c.active = (b2 > 0.0 && r2 > tol2 * b2) ? 1 : 0;
        c.nonfinite = (isfinite(b2) && isfinite(r2)) ? 0 : 1;
        if (c.nonfinite) c.active = 0;
        cgs[k] = c;
    }
}

// rr = <r, z> after a (re)start; one block per RHS
__global__ void k_cg_set_rz(CgScalars* cgs, const double* __restrict__ part, int nblk) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    if (!cgs[k].active) return;
    const double rz = row_sum(part + (int64_t)k * nblk, nblk, red);
    if (threadIdx.x == 0) {
        cgs[k].rr = rz;
        if (!isfinite(rz)) cgs[k].nonfinite = 1;
    }
}

// After a true-residual evaluation: r2true from part; converged RHS become inactive.
__global__ void k_ru_finish(CgScalars* cgs, const double* __restrict__ part, int nblk, double tol2) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    if (!cgs[k].active) return;
    const double r2 = row_sum(part + (int64_t)k * nblk, nblk, red);
    if (threadIdx.x == 0) {
        CgScalars& c = cgs[k];
        c.r2true = r2;
        c.need_ru = 0;
        if (!isfinite(r2)) { c.nonfinite = 1; c.active = 0; return; }
        if (r2 <= tol2 * c.b2) { c.active = 0; return; }
        c.r2 = r2;
        c.r2_max = r2;
    }
}

// x_hi += x_lo; x_lo = 0 (mixed mode)
__global__ void k_accum_x(double2* __restrict__ xhi, float2* __restrict__ xlo, int64_t n,
                          const CgScalars* __restrict__ cgs) {
    const int k = blockIdx.y;
    if (!cgs[k].active) return;
    const int64_t off = k * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 l = xlo[off + i];
        double2 h = xhi[off + i];
        h.x += (double)l.x;
        h.y += (double)l.y;
        xhi[off + i] = h;
        xlo[off + i] = make_float2(0.f, 0.f);
    }
}

// r = b - Ax (FP64) with partial ||r||^2; optionally also r32 = (float) r
__global__ void __launch_bounds__(256) k_residual(const double2* __restrict__ b, const double2* __restrict__ Ax,
                                                  double2* __restrict__ r, float2* __restrict__ r32, int64_t n,
                                                  double* __restrict__ part, const CgScalars* __restrict__ cgs) {
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (cgs && !cgs[k].active) return;
    const int64_t off = k * n;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 bb = b[off + i], a = Ax[off + i];
        const double2 v = make_double2(bb.x - a.x, bb.y - a.y);
        r[off + i] = v;
        if (r32) r32[off + i] = make_float2((float)v.x, (float)v.y);
        s += v.x * v.x + v.y * v.y;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

__global__ void k_to32(const double2* __restrict__ a, float2* __restrict__ b, int64_t n,
                       const CgScalars* __restrict__ cgs) {
    const int k = blockIdx.y;
    if (cgs && !cgs[k].active) return;
    const int64_t off = k * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = a[off + i];
        b[off + i] = make_float2((float)v.x, (float)v.y);
    }
}

// pnew = z + beta pold for every active right-hand side: the direction after a (re)start of
// the complex64 PCG with the fused (x, y) passes, whose iterations form it in that pass
__global__ void k_pupd(float4* __restrict__ pnew, const float4* __restrict__ z, const float4* __restrict__ pold,
                       int64_t n4, const CgScalars* __restrict__ cgs) {
    const int k = blockIdx.y;
    if (!cgs[k].active) return;
    const float beta = (float)cgs[k].beta;
    const int64_t off = k * n4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = z[off + i], b = pold[off + i];
        pnew[off + i] = make_float4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z, a.w + beta * b.w);
    }
}

__global__ void k_phi_to32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---- host driver ---------------------------------------------------------------------------
// FP64 true residual r = b - A x for the start from a guess and the reliable updates, as two
// passes through ctx->d_z64: t_ = D^dagger x, then r = b - D t_ with the complex64 copy and the
// partial norms fused into the second pass (launch_residual_D). GB300's FP64 pipe bounds both
// passes; a fused D D^dagger kernel would recompute t_ on a one-site ring around each tile (about
// 2.4 site operations per output site against 2.0 here) and measured slower (3.33 ms against 2.55
// ms for A at 80x80x160 with 8 RHS). d_z64 is dead whenever this runs: the next direction restart
// recomputes z. Right-hand sides already converged (cgs) are skipped.
static int residual64(hmc_ctx* ctx, const Lat& lat, const double* phi, const double2* x, const double2* b,
                      double2* r64, float2* r32, int nrhs, double* part, int* nblk, const CgScalars* cgs) {
    int rc;
    if ((rc = launch_apply_D<double>(ctx, lat, phi, x, ctx->d_z64, 1, nrhs, cgs))) return rc;
    return launch_residual_D(ctx, lat, phi, ctx->d_z64, b, r64, r32, nrhs, part, nblk, cgs);
}

template <typename R>
static int run(hmc_ctx* ctx, const Lat& lat, const double* phi64, const double2* b, double2* x,
               int nrhs, double tol, int maxit, int precond, hmc_cg_stats* st, bool use_x0, bool* y_ready) {
    constexpr bool kMixed = sizeof(R) == 4;
    using C = cplx<R>;
    cudaStream_t sm = ctx->stream;
    const int64_t n = 4 * lat.V;                      // complex entries per RHS
    const int64_t n16 = n * sizeof(C) / 16;
    const double tol2 = tol * tol;
    const double delta2 = 1e-6;                       // reliable update at ||r|| < 1e-3 max||r||
    CgScalars* cgs = ctx->d_cg;
    double* part = ctx->d_part;
    double* part2 = ctx->d_part + ctx->part_cap / 2;
    const dim3 vgrid(kRedBlocks, nrhs);

    C *xv, *rv, *pv, *pw, *qv, *zv;   // pv: current direction, pw: the other buffer
    const R* phiR;
    if constexpr (kMixed) {
        xv = ctx->d_x32; rv = ctx->d_r32; pv = ctx->d_p32; pw = ctx->d_p32b; qv = ctx->d_q32;
        zv = precond ? ctx->d_z32 : ctx->d_r32;
        k_phi_to32<<<(unsigned)((3 * lat.V + 255) / 256), 256, 0, sm>>>(phi64, ctx->d_phi32, 3 * lat.V);
        HMC_LAUNCH(ctx, "k_phi_to32");
        phiR = ctx->d_phi32;
        HMC_CUDA(ctx, cudaMemsetAsync(ctx->d_x32, 0, nrhs * n * sizeof(float2), sm));
    } else {
        xv = x; rv = ctx->d_r64; pv = ctx->d_p64; pw = ctx->d_p64b; qv = ctx->d_q64;
        zv = precond ? ctx->d_z64 : ctx->d_r64;
        phiR = phi64;
    }
    int rc;
    if (use_x0) {
        // start from the caller's x: ||b||^2, r_hi = b - A x (FP64) and ||r_hi||^2
        k_dot<double><<<vgrid, 256, 0, sm>>>(reinterpret_cast<const double2*>(b), reinterpret_cast<const double2*>(b),
                                             n, part2, nullptr);
        HMC_LAUNCH(ctx, "k_dot");
        int nbr = 0;
        if ((rc = residual64(ctx, lat, phi64, x, b, ctx->d_r64, kMixed ? ctx->d_r32 : nullptr, nrhs, part, &nbr,
                             nullptr)))
            return rc;
        k_cg_start<<<nrhs, 256, 0, sm>>>(cgs, part2, kRedBlocks, part, nbr, tol2);
    } else {
        // zero start: r_hi = b. t_ = D^dagger x = 0 until a true residual is formed (a right-hand
        // side with b = 0 never gets one; y_ready below covers it too)
        HMC_CUDA(ctx, cudaMemsetAsync(x, 0, nrhs * n * sizeof(double2), sm));
        if (kMixed && y_ready) HMC_CUDA(ctx, cudaMemsetAsync(ctx->d_z64, 0, nrhs * n * sizeof(double2), sm));
        k_residual<<<vgrid, 256, 0, sm>>>(b, x, ctx->d_r64, kMixed ? ctx->d_r32 : nullptr, n, part, nullptr);
        HMC_LAUNCH(ctx, "k_residual");
        k_cg_start<<<nrhs, 256, 0, sm>>>(cgs, part, kRedBlocks, nullptr, 0, tol2);
    }
    HMC_LAUNCH(ctx, "k_cg_start");

    // complex64 PCG with the fused (x, y) passes: the direction update p = z + beta p moves from
    // the operator launch into the inverse (x, y) pass (beta is known by then: <r, z> comes from
    // the tau pass)
    bool xy = false;
    if constexpr (kMixed) xy = precond && pcg_xy_path(ctx, lat);
    // directions start at zero: the first update forms p = z + 0 * p
    HMC_CUDA(ctx, cudaMemsetAsync(pv, 0, nrhs * n * sizeof(C), sm));
    if (xy) HMC_CUDA(ctx, cudaMemsetAsync(pw, 0, nrhs * n * sizeof(C), sm));
    // z = P r, rz = <r, z>
    auto restart_dir = [&]() -> int {
        if (precond) {
            if ((rc = launch_precond<R>(ctx, lat, rv, zv, nrhs, qv))) return rc;   // q is free at a restart
            k_dot<R><<<vgrid, 256, 0, sm>>>(reinterpret_cast<const V16<R>*>(rv), reinterpret_cast<const V16<R>*>(zv),
                                            n16, part, cgs);
        } else {
            k_dot<R><<<vgrid, 256, 0, sm>>>(reinterpret_cast<const V16<R>*>(rv), reinterpret_cast<const V16<R>*>(rv),
                                            n16, part, cgs);
        }
        HMC_LAUNCH(ctx, "k_dot");
        k_cg_set_rz<<<nrhs, 256, 0, sm>>>(cgs, part, kRedBlocks);
        HMC_LAUNCH(ctx, "k_cg_set_rz");
        if constexpr (kMixed) {
            if (xy) {
                // pv = z + beta pw: pw holds the direction of the last operator application
                k_pupd<<<vgrid, 256, 0, sm>>>(reinterpret_cast<float4*>(pv), reinterpret_cast<const float4*>(zv),
                                              reinterpret_cast<const float4*>(pw), n / 2, cgs);
                HMC_LAUNCH(ctx, "k_pupd");
            }
        }
        return HMC_OK;
    };
    if ((rc = restart_dir())) return rc;
    // plain complex64 CG on the strip operator: beta comes ahead of the residual update (k_cg_ab),
    // so x, r and p are updated in one pass; the first direction is p = r
    const bool fused = kMixed && !precond && strip_supported(lat);
    if (fused) HMC_CUDA(ctx, cudaMemcpyAsync(pv, rv, nrhs * n * sizeof(C), cudaMemcpyDeviceToDevice, sm));

    // true-residual update for every active RHS
    int n_ru = 0;
    auto reliable_update = [&]() -> int {
        ++n_ru;
        if constexpr (kMixed) {
            k_accum_x<<<vgrid, 256, 0, sm>>>(x, ctx->d_x32, n, cgs);
            HMC_LAUNCH(ctx, "k_accum_x");
        }
        int nbr = 0;
        if ((rc = residual64(ctx, lat, phi64, x, b, ctx->d_r64, kMixed ? ctx->d_r32 : nullptr, nrhs, part, &nbr, cgs)))
            return rc;
        k_ru_finish<<<nrhs, 256, 0, sm>>>(cgs, part, nbr, tol2);
        HMC_LAUNCH(ctx, "k_ru_finish");
        return restart_dir();
    };

    // The host reads the flags (one stream synchronisation) after at most check_every iterations.
    // From each right-hand side's residual decay it predicts when the next reliable update or the
    // stop is due and checks then, so that the last right-hand side does not run idle up to a
    // fixed multiple of check_every.
    const int check_every = 8;
    int next_check = check_every, last_check = 0;
    std::vector<double> last_r2(nrhs, -1.0), rate(nrhs, 0.0);   // ln ||r||^2 per iteration (< 0)
    auto plan_next = [&](int now) {
        int step = check_every;
        for (int k = 0; k < nrhs; ++k) {
            const CgScalars& c = ctx->h_cg[k];
            if (!c.active || !(c.r2 > 0.0)) continue;
            if (last_r2[k] > 0.0 && now > last_check && c.r2 < last_r2[k])
                rate[k] = (std::log(c.r2) - std::log(last_r2[k])) / (double)(now - last_check);
            last_r2[k] = c.r2;
            // the first threshold the residual crosses (k_cg_beta flags either)
            const double target = std::max(tol2 * c.b2, kMixed ? delta2 * c.r2_max : tol2 * c.b2);
            if (rate[k] < 0.0 && c.r2 > target) {
                const double n = (std::log(target) - std::log(c.r2)) / rate[k];
                step = std::min(step, std::max(1, (int)std::ceil(n)));
            }
        }
        last_check = now;
        next_check = now + step;
    };
    bool pending = false;   // an x update was deferred to the next iteration (fused path)
    bool done = false, nonfinite = false;
    int it = 0;
    while (!done) {
        if (it >= maxit) break;
        int nb = 0;
        if constexpr (kMixed) {
            if (xy) {
                // q = A p, partial <p, A p>; x, r update and zhat = P-hat F~^* r; beta; next p
                if ((rc = launch_apply_A<R>(ctx, lat, phiR, pv, qv, nrhs, part, &nb, cgs))) return rc;
                k_cg_alpha<<<nrhs, 256, 0, sm>>>(cgs, part, nb);
                HMC_LAUNCH(ctx, "k_cg_alpha");
                int nbr = 0, nbz = 0;
                if ((rc = launch_pcg_xy_forward(ctx, lat, xv, rv, pv, qv, zv, nrhs, cgs, part, part2, &nbr, &nbz)))
                    return rc;
                k_cg_beta<<<nrhs, 256, 0, sm>>>(cgs, part, part2, nbr, nbz, tol2, delta2, kMixed, 1, 0);
                HMC_LAUNCH(ctx, "k_cg_beta");
                if ((rc = launch_pcg_xy_inverse(ctx, lat, zv, pv, pw, nrhs, cgs))) return rc;
                { C* t = pv; pv = pw; pw = t; }
            }
        }
        if (fused) {
            if constexpr (kMixed) {
                // q = A p with <p, A p> and ||A p||^2; alpha and beta; x, r, p; ||r||^2 and the flags
                if ((rc = launch_apply_A_strip(ctx, lat, phiR, pv, qv, nrhs, part, &nb, cgs, part2))) return rc;
                k_cg_ab<<<nrhs, 256, 0, sm>>>(cgs, part, part2, nb);
                HMC_LAUNCH(ctx, "k_cg_ab");
                // x is updated on every other iteration only (see k_cg_xrp); never deferred across the
                // host's checks, where a reliable update may fold x in, nor past maxit
                const int defer = (!pending && it + 2 <= next_check && it + 2 <= maxit) ? 1 : 0;
                pending = defer != 0;
                k_cg_xrp<<<vgrid, 256, 0, sm>>>(reinterpret_cast<float4*>(xv), reinterpret_cast<float4*>(rv),
                                                reinterpret_cast<float4*>(pv), reinterpret_cast<const float4*>(qv),
                                                n16, part, cgs, defer);
                HMC_LAUNCH(ctx, "k_cg_xrp");
                k_cg_beta<<<nrhs, 256, 0, sm>>>(cgs, part, nullptr, kRedBlocks, kRedBlocks, tol2, delta2, kMixed, 0,
                                                defer);
                HMC_LAUNCH(ctx, "k_cg_beta");
            }
        } else if (!xy) {
        if (kMixed && strip_supported(lat)) {
            // p = z + beta p as a streaming pass, then q = A p on the complex64 strip kernel (the
            // operator with the update folded in has no strip form: it would stage two vectors)
            k_pupd<<<vgrid, 256, 0, sm>>>(reinterpret_cast<float4*>(pw), reinterpret_cast<const float4*>(zv),
                                          reinterpret_cast<const float4*>(pv), n / 2, cgs);
            HMC_LAUNCH(ctx, "k_pupd");
            if ((rc = launch_apply_A<R>(ctx, lat, phiR, pw, qv, nrhs, part, &nb, cgs))) return rc;
        } else {
            // p = z + beta p (fused into the operator), q = A p, partial <p, A p>
            if ((rc = launch_apply_A<R>(ctx, lat, phiR, zv, qv, nrhs, part, &nb, cgs, pv, pw))) return rc;
        }
        { C* t = pv; pv = pw; pw = t; }
        k_cg_alpha<<<nrhs, 256, 0, sm>>>(cgs, part, nb);
        HMC_LAUNCH(ctx, "k_cg_alpha");
        int nbr = kRedBlocks, nbz = kRedBlocks;
        if (precond) {
            // x += alpha p, r -= alpha q, z = P r, with ||r||^2 and <r, z>
            if ((rc = launch_cg_update_precond<R>(ctx, lat, xv, rv, pv, qv, zv, nrhs, cgs, part, part2, &nbr, &nbz)))
                return rc;
        } else {
            k_cg_xr<R><<<vgrid, 256, 0, sm>>>(reinterpret_cast<V16<R>*>(xv), reinterpret_cast<V16<R>*>(rv),
                                              reinterpret_cast<const V16<R>*>(pv), reinterpret_cast<const V16<R>*>(qv),
                                              n16, part, cgs);
            HMC_LAUNCH(ctx, "k_cg_xr");
        }
        k_cg_beta<<<nrhs, 256, 0, sm>>>(cgs, part, precond ? part2 : nullptr, nbr, nbz, tol2, delta2, kMixed, 1,
                                        0);
        HMC_LAUNCH(ctx, "k_cg_beta");
        }
        ++it;
        if (it >= next_check || it >= maxit) {
            HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_cg, cgs, nrhs * sizeof(CgScalars), cudaMemcpyDeviceToHost, sm));
            if ((rc = check_device_flags(ctx))) return rc;   // synchronises the stream
            bool any_ru = false, any_active = false;
            for (int k = 0; k < nrhs; ++k) {
                if (ctx->h_cg[k].nonfinite) nonfinite = true;
                if (ctx->h_cg[k].active) {
                    any_active = true;
                    if (ctx->h_cg[k].need_ru) any_ru = true;
                }
            }
            if (nonfinite) break;
            if (any_ru) {
                if ((rc = reliable_update())) return rc;
                HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_cg, cgs, nrhs * sizeof(CgScalars), cudaMemcpyDeviceToHost, sm));
                HMC_CUDA(ctx, cudaStreamSynchronize(sm));
                any_active = false;
                for (int k = 0; k < nrhs; ++k) {
                    if (ctx->h_cg[k].nonfinite) nonfinite = true;
                    if (ctx->h_cg[k].active) any_active = true;
                }
                if (nonfinite) break;
                for (int k = 0; k < nrhs; ++k) last_r2[k] = -1.0;   // a new cycle from the true residual
            }
            if (!any_active) done = true;
            plan_next(it);
        }
    }
    if (!done && !nonfinite) {
        // maxit reached: fold the partial solution in and measure the true residual
        if ((rc = reliable_update())) return rc;
        HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_cg, cgs, nrhs * sizeof(CgScalars), cudaMemcpyDeviceToHost, sm));
        HMC_CUDA(ctx, cudaStreamSynchronize(sm));
        done = true;
        for (int k = 0; k < nrhs; ++k)
            if (ctx->h_cg[k].active) done = false;
    }
    double worst = 0.0;
    int iters = 0;
    for (int k = 0; k < nrhs; ++k) {
        const CgScalars& c = ctx->h_cg[k];
        if (c.nonfinite) nonfinite = true;
        const double rel = c.b2 > 0.0 ? std::sqrt(c.r2true / c.b2) : 0.0;
        if (!(rel <= worst)) worst = rel;
        if (c.iters > iters) iters = c.iters;
    }
    if (st) {
        st->iterations = iters;
        st->reliable_updates = n_ru;
        st->converged = done && !nonfinite;
        st->true_rel_resid = worst;
    }
    if (nonfinite) return fail(ctx, HMC_ERR_NONFINITE, "cg_solve: non-finite residual norm");
    if (!done) return fail(ctx, HMC_ERR_NOCONV, "cg_solve: no convergence in " + std::to_string(maxit) + " iterations");
    // Mixed mode: every right-hand side stopped at a true-residual evaluation of its final x (or
    // never iterated, with t_ from the start residual or zero), and nothing else writes d_z64
    // (the preconditioned residual lives in d_z32), so d_z64 holds D^dagger x.
    if (y_ready) *y_ready = kMixed;
    return HMC_OK;
}

int cg_run(hmc_ctx* ctx, int chain, const double* phi, const double2* b, double2* x, int nrhs,
           double tol, int maxit, int precond, hmc_cg_stats* st, bool use_x0, bool* y_ready) {
    const Lat& lat = ctx->chains[chain].lat;
    if (y_ready) *y_ready = false;
    if (ctx->p.solver_mode == HMC_SOLVER_MIXED)
        return run<float>(ctx, lat, phi, b, x, nrhs, tol, maxit, precond, st, use_x0, y_ready);
    return run<double>(ctx, lat, phi, b, x, nrhs, tol, maxit, precond, st, use_x0, y_ready);
}

}  // namespace hmc
