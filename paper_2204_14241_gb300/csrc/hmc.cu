#include <algorithm>
// Context management, the C ABI of include/hmc.h, the HMC trajectory (Section "HMC":
// heatbath, momentum draw, leapfrog, Metropolis) and the Philox4x32-10 generator.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace hmc {

static thread_local std::string g_err;

int fail(hmc_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    g_err = msg;
    return code;
}

int cuda_check(hmc_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, HMC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------------------------
struct U4 { uint32_t v[4]; };

__host__ __device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) { k0 += W0; k1 += W1; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(M0, c.v[0], hi0, lo0);
        mulhilo(M1, c.v[2], hi1, lo1);
        U4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
    }
    return c;
}

__global__ void k_philox_raw(uint64_t key, U4 ctr, int64_t nblocks, uint32_t* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nblocks) return;
    // 128-bit counter + j
    U4 c = ctr;
    uint64_t lo = ((uint64_t)c.v[1] << 32 | c.v[0]);
    const uint64_t nlo = lo + (uint64_t)j;
    uint64_t hi = ((uint64_t)c.v[3] << 32 | c.v[2]) + (nlo < lo ? 1u : 0u);
    c.v[0] = (uint32_t)nlo; c.v[1] = (uint32_t)(nlo >> 32);
    c.v[2] = (uint32_t)hi; c.v[3] = (uint32_t)(hi >> 32);
    const U4 r = philox(c, (uint32_t)key, (uint32_t)(key >> 32));
#pragma unroll
    for (int q = 0; q < 4; ++q) out[4 * j + q] = r.v[q];
}

// two uniforms in (0, 1] from one Philox block (53 bits each)
__device__ __forceinline__ void uniforms(uint64_t seed, uint64_t counter, uint64_t j, double& u1, double& u2) {
    U4 c;
    c.v[0] = (uint32_t)j; c.v[1] = (uint32_t)(j >> 32);
    c.v[2] = (uint32_t)counter; c.v[3] = (uint32_t)(counter >> 32);
    const U4 r = philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t a = ((uint64_t)r.v[0] << 21) ^ (uint64_t)(r.v[1] >> 11);
    const uint64_t b = ((uint64_t)r.v[2] << 21) ^ (uint64_t)(r.v[3] >> 11);
    const double s = 1.0 / 9007199254740992.0;   // 2^-53
    u1 = ((double)(a & ((1ull << 53) - 1)) + 1.0) * s;
    u2 = ((double)(b & ((1ull << 53) - 1)) + 1.0) * s;
}

// n normals (complex_out = 0) or n complex normals with parts N(0, 1/2); Box-Muller per block.
__global__ void k_philox_normal(uint64_t seed, uint64_t counter, uint64_t jbase, int64_t n,
                                int complex_out, double* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nreal = complex_out ? 2 * n : n;
    if (2 * j >= nreal) return;
    double u1, u2;
    uniforms(seed, counter, jbase + (uint64_t)j, u1, u2);
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    const double scale = complex_out ? sqrt(0.5) : 1.0;
    out[2 * j] = scale * rad * c;
    if (2 * j + 1 < nreal) out[2 * j + 1] = scale * rad * s;
}

__global__ void k_philox_uniform(uint64_t seed, uint64_t counter, uint64_t jbase, double* out) {
    double u1, u2;
    uniforms(seed, counter, jbase, u1, u2);
    out[0] = 1.0 - u1;   // [0, 1)
}

// Metropolis test (Eq. hmc Hamiltonian) in FP64 for n chains: e[6 c + j] holds kinetic, S_B, S_PF at
// the start (j = 0, 1, 2) and at the end (j = 3, 4, 5); dH = H_end - H_start; the proposal is
// accepted when u[c] < exp(-dH) (a non-finite dH is rejected). acc[c] = 1.0 or 0.0.
__global__ void k_metropolis(const double* __restrict__ e, const double* __restrict__ u, double* __restrict__ dh,
                             double* __restrict__ acc, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double* q = e + 6 * c;
    const double h = (q[3] + q[4] + q[5]) - (q[0] + q[1] + q[2]);
    dh[c] = h;
    acc[c] = (isfinite(h) && u[c] < exp(-h)) ? 1.0 : 0.0;
}

// phi = saved phi where the proposal was rejected (*acc == 0)
__global__ void k_restore_rejected(double* __restrict__ phi, const double* __restrict__ save, int64_t n,
                                   const double* __restrict__ acc) {
    if (*acc != 0.0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        phi[i] = save[i];
}

// ---- small vector kernels ------------------------------------------------------------------
__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

// The previous solutions of a trajectory's force solves, newest first, with their weights.
constexpr int kMaxGuess = 5;   // highest extrapolation degree
struct SolHist {
    const double2* h[kMaxGuess + 1];
    double c[kMaxGuess + 1];
};

// out = sum_j c_j h_j over NP solutions (the weights come from the host); out may be one of the
// h_j. FP64 throughout: the start's error only costs iterations, but an FP32 one would sit near
// the size of the residual that a good extrapolation leaves.
template <int NP>
__global__ void __launch_bounds__(256) k_extrap(SolHist hs, double2* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) v[j] = hs.h[j][i];
        double2 s = make_double2(hs.c[0] * v[0].x, hs.c[0] * v[0].y);
#pragma unroll
        for (int j = 1; j < NP; ++j) {
            s.x = fma(hs.c[j], v[j].x, s.x);
            s.y = fma(hs.c[j], v[j].y, s.y);
        }
        out[i] = s;
    }
}

__global__ void __launch_bounds__(256) k_norm2(const double* __restrict__ a, int64_t n, double* __restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * a[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace hmc

using namespace hmc;

// ---- helpers ------------------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int check_chain(hmc_ctx* ctx, int chain) {
    if (!ctx) return fail(nullptr, HMC_ERR_ARG, "null context");
    if (chain < 0 || chain >= (int)ctx->chains.size()) return fail(ctx, HMC_ERR_ARG, "chain index out of range");
    return HMC_OK;
}

static int check_ptrs(hmc_ctx* ctx, std::initializer_list<const void*> ps) {
    for (const void* p : ps) {
        if (!p) return fail(ctx, HMC_ERR_ARG, "null pointer argument");
        if (!aligned16(p)) return fail(ctx, HMC_ERR_ARG, "pointer not 16-byte aligned");
    }
    return HMC_OK;
}

static int check_nrhs(hmc_ctx* ctx, int nrhs) {
    if (nrhs < 1 || nrhs > ctx->kmax) return fail(ctx, HMC_ERR_ARG, "nrhs must be in [1, nrhs_max]");
    return HMC_OK;
}

template <typename T> static int dalloc(hmc_ctx* ctx, T** p, int64_t count) {
    HMC_CUDA(ctx, cudaMalloc((void**)p, (size_t)count * sizeof(T)));
    return HMC_OK;
}

// m FP64 solution buffers for a degree-m chronological start
static int alloc_hist(hmc_ctx* ctx, int m, int64_t nf) {
    for (int j = 0; j < m; ++j) {
        int rc;
        if ((rc = dalloc(ctx, &ctx->d_Xhist[j], nf))) return rc;
    }
    return HMC_OK;
}

static void free_all(hmc_ctx* ctx) {
    for (double2*& b : ctx->d_Xhist) {
        cudaFree(b);
        b = nullptr;
    }
    void* ps[] = {ctx->d_r64, ctx->d_p64, ctx->d_p64b, ctx->d_p32b, ctx->d_q64, ctx->d_z64, ctx->d_X, ctx->d_pf, ctx->d_chi,
                  ctx->d_x32, ctx->d_r32, ctx->d_p32, ctx->d_q32, ctx->d_z32, ctx->d_phi32,
                  ctx->d_phi_save, ctx->d_pi, ctx->d_F, ctx->d_vel, ctx->d_z, ctx->d_fft,
                  ctx->d_part, ctx->d_red, ctx->d_cg, ctx->d_u32, ctx->d_flags};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->cap_stream = nullptr;
    batch_free(ctx);
    void* bs[] = {ctx->batch_phi32, ctx->d_energy, ctx->batch.bar, ctx->batch.iters, ctx->batch.ch};
    for (void* b : bs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    ctx->events.clear();
    if (ctx->h_cg) cudaFreeHost(ctx->h_cg);
    if (ctx->h_red) cudaFreeHost(ctx->h_red);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    free_plans(ctx);
}

int hmc::check_device_flags(hmc_ctx* ctx) {
    HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int f = ctx->h_flags[0];
    if (!f) return HMC_OK;
    HMC_CUDA(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream));
    return fail(ctx, HMC_ERR_TIMEOUT, std::string("a device-side wait gave up (flags ") + std::to_string(f) + ")");
}

// synchronise and copy `count` reduced scalars d_red[0..count) to host
static int fetch_red(hmc_ctx* ctx, int count, double* dst) {
    HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_red, ctx->d_red, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < count; ++i) dst[i] = ctx->h_red[i];
    return HMC_OK;
}

extern "C" {

const char* hmc_last_error(const hmc_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int hmc_counters(const hmc_ctx* ctx, int64_t* kernel_launches) {
    if (!ctx || !kernel_launches) return fail(nullptr, HMC_ERR_ARG, "hmc_counters: null argument");
    *kernel_launches = ctx->launches;
    return HMC_OK;
}

int hmc_init(const hmc_params* p, int n_chains, const hmc_chain* chains, void* cuda_stream, hmc_ctx** out) {
    if (!p || !out) return fail(nullptr, HMC_ERR_ARG, "hmc_init: null argument");
    *out = nullptr;
    if (n_chains < 1) return fail(nullptr, HMC_ERR_ARG, "hmc_init: n_chains must be >= 1");
    if (p->nrhs_max < 1 || p->nrhs_max > 64) return fail(nullptr, HMC_ERR_ARG, "hmc_init: nrhs_max must be in [1, 64]");
    if (p->solver_mode != HMC_SOLVER_FP64 && p->solver_mode != HMC_SOLVER_MIXED)
        return fail(nullptr, HMC_ERR_ARG, "hmc_init: unknown solver_mode");
    if (!(p->dtau > 0.0) || !(p->c > 0.0)) return fail(nullptr, HMC_ERR_ARG, "hmc_init: dtau and c must be positive");
    if (p->initial_guess < 0 || p->initial_guess > kMaxGuess)
        return fail(nullptr, HMC_ERR_ARG, "hmc_init: initial_guess must be in [0, 5]");
    hmc_ctx* ctx = new (std::nothrow) hmc_ctx();
    if (!ctx) return fail(nullptr, HMC_ERR_ARG, "hmc_init: out of host memory");
    ctx->p = *p;
    if (ctx->p.cg_tol <= 0.0) ctx->p.cg_tol = 1e-10;
    if (ctx->p.cg_maxit <= 0) ctx->p.cg_maxit = 100000;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->kmax = p->nrhs_max;
    for (int c = 0; c < n_chains; ++c) {
        const int L = chains ? chains[c].L : p->L;
        const int Nt = chains ? chains[c].Nt : p->Nt;
        const double r = chains ? chains[c].r : p->r;
        if (L < 2 || (L & 1) || L > 4096 || Nt < 2 || Nt > 65536) {
            delete ctx;
            return fail(nullptr, HMC_ERR_ARG, "hmc_init: need even L in [2, 4096] and Nt in [2, 65536]");
        }
        ChainDesc d;
        d.lat.L = L;
        d.lat.Nt = Nt;
        d.lat.V = (int64_t)Nt * L * L;
        d.r = r;
        ctx->chains.push_back(d);
        ctx->batch_off.push_back(ctx->vtot);
        ctx->vtot += d.lat.V;
        if (d.lat.V > ctx->vmax) ctx->vmax = d.lat.V;
    }
    const bool batch = p->batch_chains != 0;
    if (batch && p->solver_mode != HMC_SOLVER_MIXED) {
        delete ctx;
        return fail(nullptr, HMC_ERR_ARG, "hmc_init: batch_chains needs solver_mode HMC_SOLVER_MIXED");
    }
    ctx->tstats.assign(n_chains, hmc_traj_stats{});
    ctx->tstats_valid.assign(n_chains, 0);
    int dev = 0;
    int rc = HMC_OK;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    ctx->device = dev;
    if (e != cudaSuccess) {
        rc = cuda_check(nullptr, e, "hmc_init: device query");
        delete ctx;
        return rc;
    }
    // the batched path keeps every chain's fermion vectors and momenta live at once
    const int64_t vw = batch ? ctx->vtot : ctx->vmax;
    const int64_t nf = (int64_t)ctx->kmax * 4 * vw;   // complex entries per workspace vector
    const int64_t nb = 3 * ctx->vmax, nbw = 3 * vw;
    ctx->part_cap = 4 * (int64_t)ctx->kmax * 512;
    const int64_t need_a = (int64_t)ctx->kmax * (ctx->vmax / 16 + 1024);
    const int64_t need_m = 3 * ctx->vmax / 256 + 1024;
    if (need_a > ctx->part_cap) ctx->part_cap = need_a;
    if (need_m > ctx->part_cap) ctx->part_cap = need_m;
    const bool mixed = p->solver_mode == HMC_SOLVER_MIXED;
    if ((rc = dalloc(ctx, &ctx->d_r64, nf)) || (rc = dalloc(ctx, &ctx->d_p64, mixed ? 1 : nf)) ||
        (rc = dalloc(ctx, &ctx->d_p64b, mixed ? 1 : nf)) || (rc = dalloc(ctx, &ctx->d_p32b, mixed ? nf : 1)) ||
        (rc = dalloc(ctx, &ctx->d_q64, nf)) || (rc = dalloc(ctx, &ctx->d_z64, nf)) ||
        (rc = dalloc(ctx, &ctx->d_X, nf)) || (rc = alloc_hist(ctx, p->initial_guess, nf)) || (rc = dalloc(ctx, &ctx->d_pf, nf)) ||
        (rc = dalloc(ctx, &ctx->d_chi, nf)) || (rc = dalloc(ctx, &ctx->d_x32, mixed ? nf : 1)) ||
        (rc = dalloc(ctx, &ctx->d_r32, mixed ? nf : 1)) || (rc = dalloc(ctx, &ctx->d_p32, mixed ? nf : 1)) ||
        (rc = dalloc(ctx, &ctx->d_q32, mixed ? nf : 1)) || (rc = dalloc(ctx, &ctx->d_z32, mixed ? nf : 1)) ||
        (rc = dalloc(ctx, &ctx->d_phi32, nb)) || (rc = dalloc(ctx, &ctx->d_phi_save, nbw)) ||
        (rc = dalloc(ctx, &ctx->d_pi, nbw)) || (rc = dalloc(ctx, &ctx->d_F, nbw)) || (rc = dalloc(ctx, &ctx->d_vel, nbw)) ||
        (batch && ((rc = dalloc(ctx, &ctx->batch_phi32, 3 * ctx->vtot)) ||
                   (rc = dalloc(ctx, &ctx->d_energy, 9 * (int64_t)n_chains)) ||
                   (rc = dalloc(ctx, &ctx->batch.bar, 2)) || (rc = dalloc(ctx, &ctx->batch.iters, 4)) ||
                   (rc = dalloc(ctx, &ctx->batch.ch, n_chains)))) ||
        (rc = dalloc(ctx, &ctx->d_z, nb)) || (rc = dalloc(ctx, &ctx->d_fft, nb)) ||
        (rc = dalloc(ctx, &ctx->d_part, ctx->part_cap)) || (rc = dalloc(ctx, &ctx->d_red, 64)) ||
        (rc = dalloc(ctx, &ctx->d_cg, ctx->kmax)) || (rc = dalloc(ctx, &ctx->d_u32, 4)) ||
        (rc = dalloc(ctx, &ctx->d_flags, 16)) || (batch && (rc = batch_alloc(ctx)))) {
        std::string m = ctx->err;
        free_all(ctx);
        delete ctx;
        return fail(nullptr, rc, m);
    }
    e = cudaMallocHost((void**)&ctx->h_cg, ctx->kmax * sizeof(CgScalars));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_red, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_flags, 16 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flags, 0, 16 * sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        rc = cuda_check(nullptr, e, "hmc_init: pinned host buffers");
        free_all(ctx);
        delete ctx;
        return rc;
    }
    if ((rc = build_plans(ctx))) {
        std::string m = ctx->err;
        free_all(ctx);
        delete ctx;
        return fail(nullptr, rc, m);
    }
    *out = ctx;
    return HMC_OK;
}

int hmc_destroy(hmc_ctx* ctx) {
    if (!ctx) return HMC_OK;
    DevGuard g(ctx);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
    return HMC_OK;
}

int apply_M(hmc_ctx* ctx, int chain, int prec, const void* phi, const void* x, void* y, int dagger, int nrhs) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {phi, x, y}))) return rc;
    if (x == y) return fail(ctx, HMC_ERR_ARG, "apply_M: x and y must not overlap");
    DevGuard g(ctx);
    const Lat& lat = ctx->chains[chain].lat;
    if (prec == HMC_FP64)
        return launch_apply_D<double>(ctx, lat, (const double*)phi, (const double2*)x, (double2*)y, dagger, nrhs);
    if (prec == HMC_FP32)
        return launch_apply_D<float>(ctx, lat, (const float*)phi, (const float2*)x, (float2*)y, dagger, nrhs);
    return fail(ctx, HMC_ERR_ARG, "apply_M: unknown precision");
}

int apply_MdagM(hmc_ctx* ctx, int chain, int prec, const void* phi, const void* x, void* y, int nrhs, double* norm2) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {phi, x, y}))) return rc;
    if (x == y) return fail(ctx, HMC_ERR_ARG, "apply_MdagM: x and y must not overlap");
    DevGuard g(ctx);
    const Lat& lat = ctx->chains[chain].lat;
    double* part = norm2 ? ctx->d_part : nullptr;
    int nb = 0;
    if (prec == HMC_FP64) rc = launch_apply_A<double>(ctx, lat, (const double*)phi, (const double2*)x, (double2*)y, nrhs, part, &nb);
    else if (prec == HMC_FP32) rc = launch_apply_A<float>(ctx, lat, (const float*)phi, (const float2*)x, (float2*)y, nrhs, part, &nb);
    else return fail(ctx, HMC_ERR_ARG, "apply_MdagM: unknown precision");
    if (rc || !norm2) return rc;
    if ((rc = reduce_rows(ctx, part, nrhs, nb, ctx->d_red))) return rc;
    if ((rc = fetch_red(ctx, nrhs, norm2))) return rc;
    return check_device_flags(ctx);
}

int apply_precond(hmc_ctx* ctx, int chain, int prec, const void* x, void* y, int nrhs) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {x, y}))) return rc;
    DevGuard g(ctx);
    const Lat& lat = ctx->chains[chain].lat;
    if (prec == HMC_FP64) return launch_precond<double>(ctx, lat, (const double2*)x, (double2*)y, nrhs);
    // the FP64 q workspace (twice the bytes needed) holds the complex64 spectrum between passes
    if (prec == HMC_FP32)
        return launch_precond<float>(ctx, lat, (const float2*)x, (float2*)y, nrhs, reinterpret_cast<float2*>(ctx->d_q64));
    return fail(ctx, HMC_ERR_ARG, "apply_precond: unknown precision");
}

int cg_solve(hmc_ctx* ctx, int chain, const void* phi, const void* b, void* x, int nrhs, double tol, int maxit,
             int precond, hmc_cg_stats* st) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {phi, b, x}))) return rc;
    if (b == x) return fail(ctx, HMC_ERR_ARG, "cg_solve: b and x must not overlap");
    DevGuard g(ctx);
    if (tol <= 0.0) tol = ctx->p.cg_tol;
    if (maxit <= 0) maxit = ctx->p.cg_maxit;
    return cg_run(ctx, chain, (const double*)phi, (const double2*)b, (double2*)x, nrhs, tol, maxit, precond ? 1 : 0, st);
}

}  // extern "C"

// Per-phase GPU time of one trajectory: an event is recorded on the context's stream at every
// phase boundary, and after the trajectory's final synchronisation the time between consecutive
// events is added to the phase that started at the first of them.
struct PhaseTimer {
    hmc_ctx* ctx;
    std::vector<std::pair<int, int>> marks;   // (event index, phase starting there)
    explicit PhaseTimer(hmc_ctx* c) : ctx(c) {}
    int mark(int phase) {
        const int i = (int)marks.size();
        if (i >= (int)ctx->events.size()) {
            cudaEvent_t e;
            HMC_CUDA(ctx, cudaEventCreate(&e));
            ctx->events.push_back(e);
        }
        HMC_CUDA(ctx, cudaEventRecord(ctx->events[i], ctx->stream));
        marks.emplace_back(i, phase);
        return HMC_OK;
    }
    // call after the stream has been synchronised
    void collect(double ms[4]) {
        for (int q = 0; q < 4; ++q) ms[q] = 0.0;
        for (size_t j = 0; j + 1 < marks.size(); ++j) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ctx->events[marks[j].first], ctx->events[marks[j + 1].first]) == cudaSuccess)
                ms[marks[j].second] += t;
        }
    }
};
enum { kPhaseSolve = 0, kPhaseForce = 1, kPhaseMetric = 2, kPhaseOther = 3 };

// F, S_pf and S_b at phi for the pseudofermions pf; X receives A^{-1} pf (starting from the
// contents of X when use_x0). S_pf and S_b go to the host (s_pf, s_b) or, with dev_e, stay on the
// device as dev_e[0], dev_e[1].
static int force_impl(hmc_ctx* ctx, int chain, const double* phi, const double2* pf, int nrhs, double* F,
                      int include_boson, int precond, double* s_pf, double* s_b, hmc_cg_stats* st,
                      double2* X, bool use_x0, PhaseTimer* tm = nullptr, double* dev_e = nullptr) {
    const ChainDesc& ch = ctx->chains[chain];
    int rc;
    if (tm && (rc = tm->mark(kPhaseSolve))) return rc;
    bool y_ready = false;   // D^dagger X left by the solve's last true residual
    rc = cg_run(ctx, chain, phi, pf, X, nrhs, ctx->p.cg_tol, ctx->p.cg_maxit, precond, st, use_x0, &y_ready);
    if (rc) return rc;
    if (tm && (rc = tm->mark(kPhaseForce))) return rc;
    int nb = 0;
    if ((rc = launch_force(ctx, ch.lat, ch.r, phi, X, pf, nrhs, F, include_boson, ctx->d_part, &nb,
                           y_ready ? ctx->d_z64 : nullptr)))
        return rc;
    if (dev_e) return reduce_rows(ctx, ctx->d_part, 2, nb, dev_e);
    if (!s_pf && !s_b) return HMC_OK;
    if ((rc = reduce_rows(ctx, ctx->d_part, 2, nb, ctx->d_red))) return rc;
    double v[2];
    if ((rc = fetch_red(ctx, 2, v))) return rc;
    if (s_pf) *s_pf = v[0];
    if (s_b) *s_b = v[1];
    return HMC_OK;
}

extern "C" int force(hmc_ctx* ctx, int chain, const void* phi, const void* phi_pf, int nrhs, void* F, double* S_pf,
                     int include_boson, int precond, double* S_b, hmc_cg_stats* st) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {phi, phi_pf, F}))) return rc;
    DevGuard g(ctx);
    double sb = 0.0;
    rc = force_impl(ctx, chain, (const double*)phi, (const double2*)phi_pf, nrhs, (double*)F, include_boson,
                    precond, S_pf, (S_b || include_boson) ? &sb : nullptr, st, ctx->d_X, false);
    if (rc) return rc;
    if (S_b) {
        if (!include_boson) {
            // S_B was not part of the force pass: evaluate it separately
            int nb = 0;
            const ChainDesc& ch = ctx->chains[chain];
            if ((rc = launch_boson(ctx, ch.lat, ch.r, (const double*)phi, nullptr, ctx->d_part, &nb))) return rc;
            if ((rc = reduce_rows(ctx, ctx->d_part, 1, nb, ctx->d_red))) return rc;
            if ((rc = fetch_red(ctx, 1, &sb))) return rc;
        }
        *S_b = sb;
    }
    return HMC_OK;
}

extern "C" int metric_apply(hmc_ctx* ctx, int chain, int op, const void* sig, const void* in, void* out, double* scalar) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_ptrs(ctx, {sig, in}))) return rc;
    if (op < HMC_METRIC_MOMENTUM || op > HMC_METRIC_MNORM) return fail(ctx, HMC_ERR_ARG, "metric_apply: unknown op");
    if (op == HMC_METRIC_KINETIC || op == HMC_METRIC_MNORM) {
        if (!scalar) return fail(ctx, HMC_ERR_ARG, "metric_apply: kinetic needs a scalar output");
    } else if ((rc = check_ptrs(ctx, {out}))) {
        return rc;
    }
    DevGuard g(ctx);
    const Lat& lat = ctx->chains[chain].lat;
    if ((rc = metric_op(ctx, lat, op, (const double*)sig, (const double*)in, (double*)out, 0.0, ctx->d_red))) return rc;
    if (op == HMC_METRIC_KINETIC || op == HMC_METRIC_MNORM) return fetch_red(ctx, 1, scalar);
    return HMC_OK;
}

extern "C" int green_estimate(hmc_ctx* ctx, int chain, const void* phi, const void* v, int nrhs, void* out,
                              int precond, hmc_cg_stats* st) {
    int rc;
    if ((rc = check_chain(ctx, chain)) || (rc = check_nrhs(ctx, nrhs)) || (rc = check_ptrs(ctx, {phi, v, out}))) return rc;
    DevGuard g(ctx);
    return green_run(ctx, chain, (const double*)phi, (const double2*)v, nrhs, (double2*)out, precond ? 1 : 0, st);
}

extern "C" int philox_raw(hmc_ctx* ctx, uint64_t key, const uint32_t ctr[4], int64_t nblocks, void* out) {
    if (!ctx || !ctr || !out || nblocks < 0) return fail(ctx, HMC_ERR_ARG, "philox_raw: bad argument");
    if (nblocks == 0) return HMC_OK;
    DevGuard g(ctx);
    U4 c;
    for (int q = 0; q < 4; ++q) c.v[q] = ctr[q];
    k_philox_raw<<<(unsigned)((nblocks + 255) / 256), 256, 0, ctx->stream>>>(key, c, nblocks, (uint32_t*)out);
    HMC_LAUNCH(ctx, "k_philox_raw");
    return HMC_OK;
}

static int gen_normal(hmc_ctx* ctx, uint64_t seed, uint64_t counter, uint64_t jbase, int64_t n, int cplx, double* out) {
    const int64_t nreal = cplx ? 2 * n : n;
    const int64_t nblk = (nreal + 1) / 2;
    if (nblk == 0) return HMC_OK;
    k_philox_normal<<<(unsigned)((nblk + 255) / 256), 256, 0, ctx->stream>>>(seed, counter, jbase, n, cplx, out);
    HMC_LAUNCH(ctx, "k_philox_normal");
    return HMC_OK;
}

extern "C" int philox_normal(hmc_ctx* ctx, uint64_t seed, uint64_t counter, int64_t n, int complex_out, void* out) {
    if (!ctx || n < 0) return fail(ctx, HMC_ERR_ARG, "philox_normal: bad argument");
    int rc;
    if ((rc = check_ptrs(ctx, {out}))) return rc;
    DevGuard g(ctx);
    return gen_normal(ctx, seed, counter, 0, n, complex_out ? 1 : 0, (double*)out);
}

// ---- trajectory ----------------------------------------------------------------------------------
// d = a - b
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ d, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = a[i] - b[i];
}

static int run_chain(hmc_ctx* ctx, int c, const hmc_traj_in* in, double out_e[6], double* dH, int* acc,
                     int* iters, double* worst, double* jump2) {
    const ChainDesc& ch = ctx->chains[c];
    const Lat& lat = ch.lat;
    const int64_t nb = 3 * lat.V;
    const unsigned gb = (unsigned)((nb + 255) / 256);
    const int K = in->nrhs;
    double* phi = (double*)in->phi[c];
    const double* sig = (const double*)in->sigma_hat[c];
    cudaStream_t sm = ctx->stream;
    int rc;
    PhaseTimer tm(ctx);
    hmc_traj_stats& ts = ctx->tstats[c];
    ts = hmc_traj_stats{};
    ctx->tstats_valid[c] = 0;
    if ((rc = tm.mark(kPhaseOther))) return rc;
    HMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_phi_save, phi, nb * sizeof(double), cudaMemcpyDeviceToDevice, sm));

    // noise
    // the chain's energy record on the device: E[0..5] kinetic, S_B, S_PF at the start and at the
    // end, E[6] the uniform draw, E[7] dH, E[8] the decision
    double* E = ctx->d_red + 40;
    const double2* chi;
    const double* z;
    if (in->noise == HMC_NOISE_EXPLICIT) {
        chi = (const double2*)in->chi[c];
        z = (const double*)in->z[c];
        ctx->h_red[40] = in->u[c];
        HMC_CUDA(ctx, cudaMemcpyAsync(E + 6, ctx->h_red + 40, sizeof(double), cudaMemcpyHostToDevice, sm));
    } else {
        const uint64_t key = in->seed + 0x9E3779B97F4A7C15ull * (uint64_t)c;
        if ((rc = gen_normal(ctx, key, in->counter, 0, (int64_t)K * 4 * lat.V, 1, (double*)ctx->d_chi))) return rc;
        if ((rc = gen_normal(ctx, key, in->counter, 1ull << 48, nb, 0, ctx->d_z))) return rc;
        k_philox_uniform<<<1, 1, 0, sm>>>(key, in->counter, 2ull << 48, E + 6);
        HMC_LAUNCH(ctx, "k_philox_uniform");
        chi = ctx->d_chi;
        z = ctx->d_z;
    }

    // heatbath varphi = D chi, momentum, initial energies
    if ((rc = launch_apply_D<double>(ctx, lat, phi, chi, ctx->d_pf, 0, K))) return rc;
    if ((rc = tm.mark(kPhaseMetric))) return rc;
    if ((rc = metric_op(ctx, lat, HMC_METRIC_MOMENTUM, sig, z, ctx->d_pi, 0.0, nullptr))) return rc;
    if ((rc = metric_op(ctx, lat, HMC_METRIC_KINETIC, sig, ctx->d_pi, nullptr, 0.0, E))) return rc;
    if ((rc = tm.mark(kPhaseOther))) return rc;
    int nbb = 0;
    if ((rc = launch_boson(ctx, lat, ch.r, phi, nullptr, ctx->d_part, &nbb))) return rc;
    if ((rc = reduce_rows(ctx, ctx->d_part, 1, nbb, E + 1))) return rc;
    {
        const unsigned g = 1024;
        k_norm2<<<g, 256, 0, sm>>>((const double*)chi, (int64_t)K * 8 * lat.V, ctx->d_part);
        HMC_LAUNCH(ctx, "k_norm2");
        if ((rc = reduce_rows(ctx, ctx->d_part, 1, g, E + 2))) return rc;
    }

    // leapfrog: kick eps/2, (drift eps, kick eps) x n, last kick eps/2
    const double eps = in->eps;
    int tot_it = 0;
    double wr = 0.0;
    hmc_cg_stats st;
    // solution history (initial guesses): hist[0] the latest solution, hist[1] the one before, ...; the
    // start of the next solve is the extrapolation through the last min(nsol, mode + 1) of them,
    // built in a free buffer or in place of the oldest
    const int mode = ctx->p.initial_guess;
    double2* hist[kMaxGuess + 1] = {ctx->d_X};
    for (int j = 1; j <= mode; ++j) hist[j] = ctx->d_Xhist[j - 1];
    int nsol = 0;
    const int64_t nfv = (int64_t)K * 4 * lat.V;
    auto do_force = [&](bool want) -> int {
        const bool guess = mode && nsol >= 1;
        const int np = guess ? std::min(nsol, mode + 1) : 0;
        const int io = np < mode + 1 ? np : mode;   // free slot, or the oldest solution
        double2* xo = !guess ? hist[0] : hist[io];
        if (guess) {
            // polynomial extrapolation through np equally spaced solutions, newest first:
            // c_j = (-1)^j binomial(np, j + 1) (1; 2, -1; 3, -3, 1; 4, -6, 4, -1; ...)
            SolHist hs{};
            double cb = np;
            for (int j = 0; j < np; ++j) {
                hs.h[j] = hist[j];
                hs.c[j] = (j % 2 ? -cb : cb);
                cb = cb * (np - j - 1) / (j + 2);
            }
            const unsigned ge = (unsigned)std::min<int64_t>((nfv + 255) / 256, (int64_t)ctx->num_sms * 16);
            switch (np) {
                case 1: k_extrap<1><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
                case 2: k_extrap<2><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
                case 3: k_extrap<3><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
                case 4: k_extrap<4><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
                case 5: k_extrap<5><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
                default: k_extrap<6><<<ge, 256, 0, sm>>>(hs, xo, nfv); break;
            }
            HMC_LAUNCH(ctx, "k_extrap");
        }
        int r2 = force_impl(ctx, c, phi, ctx->d_pf, K, ctx->d_F, 1, in->precond, nullptr, nullptr, &st, xo, guess, &tm,
                            want ? ctx->d_red + 56 : nullptr);   // S_PF, S_B at the end, swapped into E below
        if (!r2) r2 = tm.mark(kPhaseOther);
        if (ts.n_solves < HMC_MAX_SOLVES) {
            ts.iterations[ts.n_solves] = st.iterations;
            ts.true_resid[ts.n_solves] = st.true_rel_resid;
        }
        ts.n_solves += 1;
        ts.reliable_updates += st.reliable_updates;
        if (guess) {
            for (int j = io; j > 0; --j) hist[j] = hist[j - 1];   // buffers past io keep their place
            hist[0] = xo;
        }
        ++nsol;
        tot_it += st.iterations;
        if (st.true_rel_resid > wr) wr = st.true_rel_resid;
        return r2;
    };
    rc = do_force(false);
    if (!rc) {
        k_axpy<<<gb, 256, 0, sm>>>(0.5 * eps, ctx->d_F, ctx->d_pi, nb);
        HMC_LAUNCH(ctx, "k_axpy");
        for (int i = 1; i <= in->n_leap && !rc; ++i) {
            if ((rc = tm.mark(kPhaseMetric))) break;
            if ((rc = metric_op(ctx, lat, HMC_METRIC_VELOCITY, sig, ctx->d_pi, phi, eps, nullptr))) break;
            if ((rc = do_force(i == in->n_leap))) break;
            k_axpy<<<gb, 256, 0, sm>>>(i < in->n_leap ? eps : 0.5 * eps, ctx->d_F, ctx->d_pi, nb);
            HMC_LAUNCH(ctx, "k_axpy");
        }
        if (in->n_leap == 0 && !rc) rc = do_force(true);
    }
    if (!rc) rc = tm.mark(kPhaseMetric);
    if (!rc) rc = metric_op(ctx, lat, HMC_METRIC_KINETIC, sig, ctx->d_pi, nullptr, 0.0, E + 3);
    if (!rc) rc = tm.mark(kPhaseOther);
    if (!rc && jump2) {
        // squared M-norm of the proposed jump (Eq. ESJD), accepted or not
        k_sub<<<gb, 256, 0, sm>>>(phi, ctx->d_phi_save, ctx->d_vel, nb);
        HMC_LAUNCH(ctx, "k_sub");
        rc = metric_op(ctx, lat, HMC_METRIC_MNORM, sig, ctx->d_vel, nullptr, 0.0, ctx->d_red + 60);
    }
    *iters = tot_it;
    *worst = wr;
    if (rc) {
        cudaMemcpyAsync(phi, ctx->d_phi_save, nb * sizeof(double), cudaMemcpyDeviceToDevice, sm);
        cudaStreamSynchronize(sm);
        return rc;
    }
    // the Metropolis test and the restore of a rejected proposal on the device
    HMC_CUDA(ctx, cudaMemcpyAsync(E + 4, ctx->d_red + 57, sizeof(double), cudaMemcpyDeviceToDevice, sm));   // S_B
    HMC_CUDA(ctx, cudaMemcpyAsync(E + 5, ctx->d_red + 56, sizeof(double), cudaMemcpyDeviceToDevice, sm));   // S_PF
    k_metropolis<<<1, 32, 0, sm>>>(E, E + 6, E + 7, E + 8, 1);
    HMC_LAUNCH(ctx, "k_metropolis");
    k_restore_rejected<<<(unsigned)std::min<int64_t>(gb, (int64_t)ctx->num_sms * 8), 256, 0, sm>>>(phi, ctx->d_phi_save,
                                                                                                   nb, E + 8);
    HMC_LAUNCH(ctx, "k_restore_rejected");
    if ((rc = tm.mark(kPhaseOther))) return rc;
    HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_red, E, 9 * sizeof(double), cudaMemcpyDeviceToHost, sm));
    if (jump2) HMC_CUDA(ctx, cudaMemcpyAsync(ctx->h_red + 9, ctx->d_red + 60, sizeof(double), cudaMemcpyDeviceToHost, sm));
    HMC_CUDA(ctx, cudaStreamSynchronize(sm));
    for (int q = 0; q < 6; ++q) out_e[q] = ctx->h_red[q];
    *dH = ctx->h_red[7];
    *acc = ctx->h_red[8] != 0.0 ? 1 : 0;
    if (jump2) *jump2 = ctx->h_red[9];
    if (!std::isfinite(*dH)) return fail(ctx, HMC_ERR_NONFINITE, "trajectory: non-finite energy change");
    tm.collect(ts.phase_ms);
    ctx->tstats_valid[c] = 1;
    return HMC_OK;
}

extern "C" int hmc_bounds_status(unsigned int* word, int* enabled) {
    if (!word) return fail(nullptr, HMC_ERR_ARG, "hmc_bounds_status: null argument");
#ifdef HMC_BOUNDS
    if (enabled) *enabled = 1;
#else
    if (enabled) *enabled = 0;
#endif
    *word = bounds_take_stencil() | bounds_take_strip();
    return HMC_OK;
}

extern "C" int hmc_trajectory_stats(const hmc_ctx* ctx, int chain, hmc_traj_stats* out) {
    if (!ctx || !out) return fail(nullptr, HMC_ERR_ARG, "hmc_trajectory_stats: null argument");
    if (chain < 0 || chain >= (int)ctx->chains.size())
        return fail(nullptr, HMC_ERR_ARG, "hmc_trajectory_stats: chain index out of range");
    if (!ctx->tstats_valid[chain]) return fail(nullptr, HMC_ERR_STATE, "hmc_trajectory_stats: no completed trajectory");
    *out = ctx->tstats[chain];
    return HMC_OK;
}

// One HMC update of every chain together (hmc_params.batch_chains): the same steps as run_chain,
// with the per-chain work issued back to back without host synchronisation and every force solve
// of all chains in one persistent launch (batched_cg). Concatenated layouts: fermion vectors
// [chain][k][V_c][4] at item offset K off_c, boson fields [chain][3][V_c] at 3 off_c. The host
// synchronises once, for the energies and the Metropolis decisions.
static int run_batched(hmc_ctx* ctx, const hmc_traj_in* in, hmc_traj_out* out) {
    const int nc = (int)ctx->chains.size();
    const int K = in->nrhs;
    cudaStream_t sm = ctx->stream;
    int rc;
    PhaseTimer tm(ctx);
    if ((rc = tm.mark(kPhaseOther))) return rc;
    for (int c = 0; c < nc; ++c) {
        ctx->tstats[c] = hmc_traj_stats{};
        ctx->tstats_valid[c] = 0;
    }
    auto fvec = [&](double2* base, int c) { return base + (int64_t)K * 4 * ctx->batch_off[c]; };
    auto bvec = [&](double* base, int c) { return base + 3 * ctx->batch_off[c]; };
    std::vector<const double*> phis(nc);
    // [6 c + j]: kinetic, S_B, S_PF at start and end; [6 nc + c]: uniform draw; [7 nc + c]: dH;
    // [8 nc + c]: the Metropolis decision
    double* E = ctx->d_energy;
    // heatbath, momenta, initial energies
    for (int c = 0; c < nc; ++c) {
        const Lat& lat = ctx->chains[c].lat;
        const int64_t nb = 3 * lat.V;
        double* phi = (double*)in->phi[c];
        phis[c] = phi;
        HMC_CUDA(ctx, cudaMemcpyAsync(bvec(ctx->d_phi_save, c), phi, nb * sizeof(double), cudaMemcpyDeviceToDevice, sm));
        const double2* chi;
        const double* z;
        if (in->noise == HMC_NOISE_EXPLICIT) {
            chi = (const double2*)in->chi[c];
            z = (const double*)in->z[c];
            HMC_CUDA(ctx, cudaMemcpyAsync(E + 6 * nc + c, in->u + c, sizeof(double), cudaMemcpyHostToDevice, sm));
        } else {
            const uint64_t key = in->seed + 0x9E3779B97F4A7C15ull * (uint64_t)c;
            if ((rc = gen_normal(ctx, key, in->counter, 0, (int64_t)K * 4 * lat.V, 1, (double*)ctx->d_chi))) return rc;
            if ((rc = gen_normal(ctx, key, in->counter, 1ull << 48, nb, 0, ctx->d_z))) return rc;
            k_philox_uniform<<<1, 1, 0, sm>>>(key, in->counter, 2ull << 48, E + 6 * nc + c);
            HMC_LAUNCH(ctx, "k_philox_uniform");
            chi = ctx->d_chi;
            z = ctx->d_z;
        }
        if ((rc = launch_apply_D<double>(ctx, lat, phi, chi, fvec(ctx->d_pf, c), 0, K))) return rc;
        k_norm2<<<1024, 256, 0, sm>>>((const double*)chi, (int64_t)K * 8 * lat.V, ctx->d_part);
        HMC_LAUNCH(ctx, "k_norm2");
        if ((rc = reduce_rows(ctx, ctx->d_part, 1, 1024, E + 6 * c + 2))) return rc;
        const double* sig = (const double*)in->sigma_hat[c];
        if ((rc = metric_op(ctx, lat, HMC_METRIC_MOMENTUM, sig, z, bvec(ctx->d_pi, c), 0.0, nullptr))) return rc;
        if ((rc = metric_op(ctx, lat, HMC_METRIC_KINETIC, sig, bvec(ctx->d_pi, c), nullptr, 0.0, E + 6 * c))) return rc;
        int nbb = 0;
        if ((rc = launch_boson(ctx, lat, ctx->chains[c].r, phi, nullptr, ctx->d_part, &nbb))) return rc;
        if ((rc = reduce_rows(ctx, ctx->d_part, 1, nbb, E + 6 * c + 1))) return rc;
    }
    // leapfrog with the chronological start over the concatenated solutions; every solve records
    // its statistics on the device (slot = solve index) and nothing in it waits for the host, so
    // with batch_graph the whole leapfrog is captured once and replayed as a CUDA graph
    if ((rc = batched_begin(ctx, K, phis.data()))) return rc;
    const int mode = ctx->p.initial_guess;
    double2* hist[kMaxGuess + 1] = {ctx->d_X};
    for (int j = 1; j <= mode; ++j) hist[j] = ctx->d_Xhist[j - 1];
    int nsol = 0;
    const int64_t nall = (int64_t)K * 4 * ctx->vtot;
    bool capturing = false;
    auto mark = [&](int phase) -> int { return capturing ? HMC_OK : tm.mark(phase); };
    auto do_force = [&](bool want) -> int {
        const bool guess = mode && nsol >= 1;
        const int np = guess ? std::min(nsol, mode + 1) : 0;
        const int io = np < mode + 1 ? np : mode;
        double2* xo = !guess ? hist[0] : hist[io];
        if (guess) {
            SolHist hs{};
            double cb = np;
            for (int j = 0; j < np; ++j) {
                hs.h[j] = hist[j];
                hs.c[j] = (j % 2 ? -cb : cb);
                cb = cb * (np - j - 1) / (j + 2);
            }
            const unsigned ge = (unsigned)std::min<int64_t>((nall + 255) / 256, (int64_t)ctx->num_sms * 16);
            switch (np) {
                case 1: k_extrap<1><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
                case 2: k_extrap<2><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
                case 3: k_extrap<3><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
                case 4: k_extrap<4><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
                case 5: k_extrap<5><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
                default: k_extrap<6><<<ge, 256, 0, sm>>>(hs, xo, nall); break;
            }
            HMC_LAUNCH(ctx, "k_extrap");
        }
        int r2;
        if ((r2 = mark(kPhaseSolve))) return r2;
        if ((r2 = batched_solve(ctx, K, ctx->d_pf, xo, guess, ctx->p.cg_tol, ctx->p.cg_maxit, nsol))) return r2;
        if ((r2 = mark(kPhaseForce))) return r2;
        for (int c = 0; c < nc; ++c) {
            const ChainDesc& ch = ctx->chains[c];
            int nb = 0;
            // D^dagger X of the solution is left in d_z64 by the batched solve
            if ((r2 = launch_force(ctx, ch.lat, ch.r, phis[c], fvec(xo, c), fvec(ctx->d_pf, c), K, bvec(ctx->d_F, c), 1,
                                   ctx->d_part, &nb, fvec(ctx->d_z64, c))))
                return r2;
            if (want) {
                if ((r2 = reduce_rows(ctx, ctx->d_part, 1, nb, E + 6 * c + 5))) return r2;
                if ((r2 = reduce_rows(ctx, ctx->d_part + nb, 1, nb, E + 6 * c + 4))) return r2;
            }
        }
        if ((r2 = mark(kPhaseOther))) return r2;
        if (guess) {
            for (int j = io; j > 0; --j) hist[j] = hist[j - 1];
            hist[0] = xo;
        }
        ++nsol;
        return HMC_OK;
    };
    const double eps = in->eps;
    const int64_t nball = 3 * ctx->vtot;
    const unsigned gball = (unsigned)((nball + 255) / 256);
    auto leapfrog = [&]() -> int {
        int r2 = do_force(in->n_leap == 0);
        if (r2) return r2;
        k_axpy<<<gball, 256, 0, sm>>>(0.5 * eps, ctx->d_F, ctx->d_pi, nball);
        HMC_LAUNCH(ctx, "k_axpy");
        for (int i = 1; i <= in->n_leap; ++i) {
            if ((r2 = mark(kPhaseMetric))) return r2;
            for (int c = 0; c < nc; ++c)
                if ((r2 = metric_op(ctx, ctx->chains[c].lat, HMC_METRIC_VELOCITY, (const double*)in->sigma_hat[c],
                                    bvec(ctx->d_pi, c), (double*)in->phi[c], eps, nullptr)))
                    return r2;
            if ((r2 = mark(kPhaseOther))) return r2;
            if ((r2 = do_force(i == in->n_leap))) return r2;
            k_axpy<<<gball, 256, 0, sm>>>(i < in->n_leap ? eps : 0.5 * eps, ctx->d_F, ctx->d_pi, nball);
            HMC_LAUNCH(ctx, "k_axpy");
        }
        return HMC_OK;
    };
    if (ctx->p.batch_graph) {
        // the graph is valid for these settings and buffers (everything else it touches is the
        // context's own workspace)
        std::vector<unsigned long long> key;
        auto bits = [](double v) { unsigned long long u; memcpy(&u, &v, 8); return u; };
        key.push_back((unsigned long long)in->n_leap);
        key.push_back(bits(eps));
        key.push_back((unsigned long long)K);
        key.push_back((unsigned long long)mode);
        key.push_back(bits(ctx->p.cg_tol));
        key.push_back((unsigned long long)ctx->p.cg_maxit);
        key.push_back((unsigned long long)ctx->p.test_wait_timeout);
        key.push_back((unsigned long long)ctx->p.wait_spin_limit);
        for (int c = 0; c < nc; ++c) {
            key.push_back((unsigned long long)(uintptr_t)in->phi[c]);
            key.push_back((unsigned long long)(uintptr_t)in->sigma_hat[c]);
        }
        if (!ctx->bgraph || key != ctx->bgraph_key) {
            if (ctx->bgraph) {
                cudaGraphExecDestroy(ctx->bgraph);
                ctx->bgraph = nullptr;
            }
            // capture on the context's own non-blocking stream (the legacy default stream, which a
            // caller may have given hmc_init, cannot be captured); the graph runs on ctx->stream
            if (!ctx->cap_stream) HMC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaStream_t home = ctx->stream;
            HMC_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            const int64_t l0 = ctx->launches;
            ctx->stream = sm = ctx->cap_stream;
            capturing = true;
            rc = leapfrog();
            capturing = false;
            ctx->stream = sm = home;
            ctx->bgraph_kernels = ctx->launches - l0;   // counted again at every replay
            ctx->launches = l0;
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (!rc && ec != cudaSuccess)
                rc = fail(ctx, HMC_ERR_CUDA, std::string("trajectory: graph capture: ") + cudaGetErrorString(ec));
            if (!rc) {
                const cudaError_t ei = cudaGraphInstantiate(&ctx->bgraph, graph, 0);
                if (ei != cudaSuccess) {
                    ctx->bgraph = nullptr;
                    rc = fail(ctx, HMC_ERR_CUDA, std::string("trajectory: graph instantiation: ") +
                                                     cudaGetErrorString(ei));
                }
            }
            if (graph) cudaGraphDestroy(graph);
            if (rc) {
                cudaGetLastError();
                return rc;
            }
            ctx->bgraph_key = key;
        } else {
            nsol = in->n_leap + 1;   // what the captured leapfrog performs
        }
        if ((rc = tm.mark(kPhaseSolve))) return rc;
        HMC_CUDA(ctx, cudaGraphLaunch(ctx->bgraph, sm));
        ctx->launches += ctx->bgraph_kernels;
        if ((rc = tm.mark(kPhaseOther))) return rc;
    } else {
        rc = leapfrog();
    }
    // statistics of every solve, read once
    std::vector<int> its((size_t)std::max(nsol, 1) * nc, 0), nru(std::max(nsol, 1), 0);
    std::vector<double> wres((size_t)std::max(nsol, 1) * nc, 0.0);
    std::vector<int> tot_it(nc, 0);
    std::vector<double> worst(nc, 0.0);
    if (!rc) rc = batched_collect(ctx, K, nsol, its.data(), wres.data(), nru.data());
    if (!rc) {
        const int kept = std::min(nsol, HMC_MAX_SOLVES);
        for (int j = 0; j < kept; ++j) {
            for (int c = 0; c < nc; ++c) {
                hmc_traj_stats& ts = ctx->tstats[c];
                ts.iterations[j] = its[(size_t)j * nc + c];
                ts.true_resid[j] = wres[(size_t)j * nc + c];
                ts.reliable_updates += nru[j];
                tot_it[c] += its[(size_t)j * nc + c];
                worst[c] = std::max(worst[c], wres[(size_t)j * nc + c]);
            }
        }
        for (int c = 0; c < nc; ++c) ctx->tstats[c].n_solves = nsol;
    }
    if (!rc) rc = tm.mark(kPhaseMetric);
    for (int c = 0; c < nc && !rc; ++c) {
        rc = metric_op(ctx, ctx->chains[c].lat, HMC_METRIC_KINETIC, (const double*)in->sigma_hat[c], bvec(ctx->d_pi, c),
                       nullptr, 0.0, E + 6 * c + 3);
        if (!rc && out && out->jump2) {
            const Lat& lat = ctx->chains[c].lat;
            const int64_t nb = 3 * lat.V;
            k_sub<<<(unsigned)((nb + 255) / 256), 256, 0, sm>>>(phis[c], bvec(ctx->d_phi_save, c), ctx->d_vel, nb);
            HMC_LAUNCH(ctx, "k_sub");
            rc = metric_op(ctx, lat, HMC_METRIC_MNORM, (const double*)in->sigma_hat[c], ctx->d_vel, nullptr, 0.0,
                           ctx->d_red + c % 64);
            if (!rc) HMC_CUDA(ctx, cudaMemcpyAsync(out->jump2 + c, ctx->d_red + c % 64, sizeof(double),
                                                   cudaMemcpyDeviceToHost, sm));
        }
    }
    if (!rc) rc = tm.mark(kPhaseOther);
    // the Metropolis test of every chain and the restore of rejected proposals on the device
    if (!rc) {
        k_metropolis<<<(unsigned)((nc + 127) / 128), 128, 0, sm>>>(E, E + 6 * nc, E + 7 * nc, E + 8 * nc, nc);
        HMC_LAUNCH(ctx, "k_metropolis");
    }
    for (int c = 0; c < nc; ++c) {
        const int64_t nb = 3 * ctx->chains[c].lat.V;
        if (!rc) {
            k_restore_rejected<<<(unsigned)std::min<int64_t>((nb + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, sm>>>(
                (double*)in->phi[c], bvec(ctx->d_phi_save, c), nb, E + 8 * nc + c);
            HMC_LAUNCH(ctx, "k_restore_rejected");
        } else {
            HMC_CUDA(ctx, cudaMemcpyAsync((double*)in->phi[c], bvec(ctx->d_phi_save, c), nb * sizeof(double),
                                          cudaMemcpyDeviceToDevice, sm));
        }
    }
    std::vector<double> he(9 * nc, 0.0);
    if (!rc) {
        HMC_CUDA(ctx, cudaMemcpyAsync(he.data(), E, 9 * nc * sizeof(double), cudaMemcpyDeviceToHost, sm));
        HMC_CUDA(ctx, cudaStreamSynchronize(sm));
    }
    int first_err = rc;
    for (int c = 0; c < nc; ++c) {
        const double h = rc ? 0.0 : he[7 * nc + c];
        const int acc = (!rc && he[8 * nc + c] != 0.0) ? 1 : 0;
        if (!rc && !std::isfinite(h) && !first_err)
            first_err = fail(ctx, HMC_ERR_NONFINITE, "trajectory: non-finite energy change");
        if (out) {
            if (out->dH) out->dH[c] = h;
            if (out->accepted) out->accepted[c] = acc;
            if (out->energies) for (int q = 0; q < 6; ++q) out->energies[6 * c + q] = rc ? 0.0 : he[6 * c + q];
            if (out->cg_iterations) out->cg_iterations[c] = tot_it[c];
            if (out->max_true_resid) out->max_true_resid[c] = worst[c];
        }
    }
    if ((rc = tm.mark(kPhaseOther)) && !first_err) first_err = rc;
    HMC_CUDA(ctx, cudaStreamSynchronize(sm));
    double ms[4];
    tm.collect(ms);
    for (int c = 0; c < nc; ++c) {
        for (int q = 0; q < 4; ++q) ctx->tstats[c].phase_ms[q] = ms[q];   // phases shared by all chains
        ctx->tstats_valid[c] = first_err ? 0 : 1;
    }
    return first_err;
}

extern "C" int trajectory(hmc_ctx* ctx, const hmc_traj_in* in, hmc_traj_out* out) {
    if (!ctx || !in) return fail(ctx, HMC_ERR_ARG, "trajectory: null argument");
    int rc;
    if ((rc = check_nrhs(ctx, in->nrhs))) return rc;
    if (in->n_leap < 0 || !(in->eps >= 0.0)) return fail(ctx, HMC_ERR_ARG, "trajectory: bad eps or n_leap");
    if (!in->phi || !in->sigma_hat) return fail(ctx, HMC_ERR_ARG, "trajectory: null phi or sigma_hat array");
    if (in->noise != HMC_NOISE_EXPLICIT && in->noise != HMC_NOISE_PHILOX) return fail(ctx, HMC_ERR_ARG, "trajectory: unknown noise mode");
    if (in->noise == HMC_NOISE_EXPLICIT && (!in->chi || !in->z || !in->u))
        return fail(ctx, HMC_ERR_ARG, "trajectory: explicit noise needs chi, z and u");
    const int nc = (int)ctx->chains.size();
    for (int c = 0; c < nc; ++c) {
        if ((rc = check_ptrs(ctx, {in->phi[c], in->sigma_hat[c]}))) return rc;
        if (in->noise == HMC_NOISE_EXPLICIT && (rc = check_ptrs(ctx, {in->chi[c], in->z[c]}))) return rc;
    }
    DevGuard g(ctx);
    if (ctx->p.batch_chains) return run_batched(ctx, in, out);
    int first_err = HMC_OK;
    for (int c = 0; c < nc; ++c) {
        double e[6] = {0, 0, 0, 0, 0, 0}, dh = 0.0, worst = 0.0, j2 = 0.0;
        int acc = 0, it = 0;
        rc = run_chain(ctx, c, in, e, &dh, &acc, &it, &worst, (out && out->jump2) ? &j2 : nullptr);
        if (rc && !first_err) first_err = rc;
        if (out) {
            if (out->dH) out->dH[c] = dh;
            if (out->accepted) out->accepted[c] = acc;
            if (out->energies) for (int q = 0; q < 6; ++q) out->energies[6 * c + q] = e[q];
            if (out->cg_iterations) out->cg_iterations[c] = it;
            if (out->max_true_resid) out->max_true_resid[c] = worst;
            if (out->jump2) out->jump2[c] = j2;
        }
    }
    return first_err;
}
