// Host-side context and cross-file kernel launchers of libhmc.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "common.cuh"

namespace hmc {

struct FftPlan {
    int n = 0;
    std::vector<int> radix;      // factors, applied in order
    double2* tw64 = nullptr;     // e^{-2 pi i k / n}, k < n (device)
    float2* tw32 = nullptr;
};

struct PcTables {
    int L = 0, Nt = 0;
    double* cosk = nullptr;     // cos(2 pi m / L)
    double2* eitw = nullptr;    // e^{i w_n}, w_n = (2n + 1) pi / Nt
    double2* twist = nullptr;   // e^{i pi t / Nt}
    float* cosk32 = nullptr;    // float copies for the FP32 path
    float2* eitw32 = nullptr;
    float2* twist32 = nullptr;
    float* cosk32_xy = nullptr; // cos(2 pi k(m) / L), k(m) the frequency at position m after the (x, y) pass
    float2* eitw32_tau = nullptr;   // e^{i w_n(p)}, n(p) the frequency at position p inside the in-place tau pass
};

// Tile shape chosen for the fused A kernel per (L, Nt, nrhs, precision).
// Block schedule of the strip operator for one (lattice, nrhs, resident blocks): right-hand side
// k runs in nch[k] time chunks of its Nt slices; blocks are launched right-hand side by right-hand
// side in the order `order`, chunk by chunk, the strips of a chunk together.
struct StripSched {
    int L = 0, Nt = 0, nrhs = 0, slots = 0;   // key: lattice, right-hand sides, resident blocks
    int maxch = 0;                             // largest chunk count (partial-sum stride / strips)
    int nblk = 0;                              // blocks of the launch
    unsigned char order[64];
    unsigned char nch[64];
};

struct ATuned {
    int L, Nt, nrhs, prec;
    int TX, TY, C;
};

struct ChainDesc {
    Lat lat;
    double r;
};

// Chain table of the batched solve (batch.cu): geometry, item offset of the chain's K
// right-hand sides in the concatenated vectors, and its fields.
struct BChainDev {
    int L, Nt, LL;
    float invL, invLL;
    int64_t V;
    int64_t off;
    const double* phi64;
    const float* phi32;
};

// Device state of the batched solve, built on first use for a right-hand-side count.
struct BatchWork {
    int K = 0, ntiles = 0, grid = 0;
    int kcap = 0, ntiles_cap = 0;   // capacities allocated at hmc_init (nrhs_max right-hand sides)
    void* tiles = nullptr;      // tile table
    int* pair_t0 = nullptr;     // first tile of each (chain, RHS) pair
    void* sc = nullptr;         // per-pair solver scalars
    double* part = nullptr;     // per-tile partial sums
    unsigned* bar = nullptr;    // grid barrier words
    int* iters = nullptr;       // [0] iterations of the slowest pair, [1] reliable updates, [2] active pairs
    BChainDev* ch = nullptr;    // chain table (n_chains entries)
    void* hist = nullptr;       // per-solve statistics of every pair, HMC_MAX_SOLVES solves of a trajectory
    int* hist_ru = nullptr;     // reliable updates of each solve
    std::vector<BChainDev> hch; // host copy of the chain table of the current trajectory
};

// Per-RHS solver scalars, device resident (kernels read alpha/beta from here).
struct CgScalars {
    double rr;        // <r, z> (or <r, r> without preconditioner) of the current iterate
    double rr_new;
    double pAp;
    double alpha;
    double beta;
    double r2;        // <r, r> (stopping test)
    double r2_max;    // largest ||r||^2 since the last reliable update
    double b2;        // <b, b>
    double r2true;    // ||b - A x||^2 at the last true-residual evaluation
    double carry;     // fused plain CG: alpha / beta of an iteration whose x update was deferred
    int active;       // 1 while this RHS iterates
    int iters;
    int need_ru;      // set when a true-residual (reliable) update is due
    int nonfinite;    // set when a norm is NaN or Inf
};

}  // namespace hmc

struct hmc_ctx {
    hmc_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;               // CUDA device current at hmc_init; every entry point runs on it
    std::vector<hmc::ChainDesc> chains;
    int64_t vmax = 0;
    int kmax = 1;
    std::string err;
    int num_sms = 0;
    int64_t launches = 0;         // kernels launched (tracing)

    // FFT plans keyed by length
    std::vector<hmc::FftPlan> plans;
    std::vector<hmc::PcTables> pcs;
    std::vector<hmc::ATuned> atuned;   // tile shapes picked for the fused A kernel
    std::vector<hmc::StripSched> strip_sched;   // block schedules of the strip operator
    cudaGraphExec_t bgraph = nullptr;           // batched leapfrog graph (hmc_params.batch_graph)
    std::vector<unsigned long long> bgraph_key; // what it was captured for
    int64_t bgraph_kernels = 0;                 // kernel launches in it
    cudaStream_t cap_stream = nullptr;          // private stream the graph is captured on
    hmc::BatchWork batch;                 // batched solve (hmc_params.batch_chains)
    std::vector<int64_t> batch_off;       // site offset of each chain in the concatenated fields
    int64_t vtot = 0;                     // sum of the chains' volumes
    float* batch_phi32 = nullptr;         // FP32 copies of every chain's phi, concatenated
    double* d_energy = nullptr;           // per chain: 6 energies and the Metropolis uniform
    std::vector<hmc_traj_stats> tstats;   // per chain: record of its last trajectory
    std::vector<int> tstats_valid;
    std::vector<cudaEvent_t> events;      // pool for the per-phase timing of trajectory()

    // fermion workspace (complex, K * 4 * vmax entries each)
    double2* d_r64 = nullptr;     // FP64 residual / true residual
    double2* d_p64 = nullptr;
    double2* d_p64b = nullptr;    // second direction buffer (ping-pong)
    double2* d_q64 = nullptr;
    double2* d_z64 = nullptr;
    double2* d_X = nullptr;       // solve output used by force
    double2* d_Xhist[5] = {};     // earlier solutions of a trajectory (chronological initial guess)
    double2* d_pf = nullptr;      // pseudofermion fields of a trajectory
    double2* d_chi = nullptr;     // heatbath noise (Philox mode)
    float2* d_x32 = nullptr;
    float2* d_r32 = nullptr;
    float2* d_p32 = nullptr;
    float2* d_p32b = nullptr;
    float2* d_q32 = nullptr;
    float2* d_z32 = nullptr;
    float* d_phi32 = nullptr;     // 3 * vmax

    // boson workspace (3 * vmax doubles each)
    double* d_phi_save = nullptr;
    double* d_pi = nullptr;
    double* d_F = nullptr;
    double* d_vel = nullptr;
    double* d_z = nullptr;
    double2* d_fft = nullptr;     // 3 * vmax complex128

    // reductions
    double* d_part = nullptr;     // partial sums, part_cap doubles
    int64_t part_cap = 0;
    double* d_red = nullptr;      // reduced scalars, 64 doubles
    hmc::CgScalars* d_cg = nullptr;   // kmax entries
    hmc::CgScalars* h_cg = nullptr;   // pinned mirror
    double* h_red = nullptr;          // pinned, 64 doubles
    uint32_t* d_u32 = nullptr;        // 4 words scratch for uniforms
    int* d_flags = nullptr;           // device error word [0]: bit 0 a bounded wait gave up, bit 1 its drain did too
    int* h_flags = nullptr;           // pinned mirror

};

namespace hmc {

// cudaFuncSetAttribute applies to the current device only, so each kernel remembers, per device
// ordinal, whether its attribute has been set there (ordinals >= 64 set it on every call).
struct PerDevice {
    std::atomic<uint64_t> done{0};
    bool pending(uint64_t* bit) {
        int d = 0;
        *bit = 0;
        if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return true;
        *bit = 1ull << d;
        return (done.load(std::memory_order_acquire) & *bit) == 0;
    }
    void mark(uint64_t bit) { done.fetch_or(bit, std::memory_order_acq_rel); }
};

// Makes the context's device current for the lifetime of the guard and restores the caller's.
struct DevGuard {
    int prev = -1;
    explicit DevGuard(const hmc_ctx* ctx) {
        int cur = 0;
        if (ctx && cudaGetDevice(&cur) == cudaSuccess && cur != ctx->device && cudaSetDevice(ctx->device) == cudaSuccess)
            prev = cur;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DevGuard(const DevGuard&) = delete;
    DevGuard& operator=(const DevGuard&) = delete;
};

// status helpers
int fail(hmc_ctx* ctx, int code, const std::string& msg);
int cuda_check(hmc_ctx* ctx, cudaError_t e, const char* what);
#define HMC_CUDA(ctx, call)                                              \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::hmc::cuda_check(ctx, _e, #call); \
    } while (0)
#define HMC_LAUNCH(ctx, what)                                             \
    do {                                                                  \
        ++(ctx)->launches;                                                \
        cudaError_t _e = cudaGetLastError();                              \
        if (_e != cudaSuccess) return ::hmc::cuda_check(ctx, _e, what);   \
    } while (0)

template <typename R> Coef<R> make_coef(const hmc_params& p);

// stencil.cu
// y = D x (dagger 0) or D^dagger x; right-hand sides with cgs[k].active == 0 are skipped when cgs
// is given.
template <typename R>
int launch_apply_D(hmc_ctx* ctx, const Lat& lat, const R* phi, const cplx<R>* x, cplx<R>* y,
                   int dagger, int nrhs, const CgScalars* cgs = nullptr);
// FP64 true residual r = b - D t (t = D^dagger x from launch_apply_D), written as r64 and, if
// r32 != nullptr, as complex64; per-block partial sums of ||r||^2 in part[k * nblk + b], nblk =
// *nblk_out. Inactive right-hand sides (cgs) are skipped.
int launch_residual_D(hmc_ctx* ctx, const Lat& lat, const double* phi, const double2* t, const double2* b,
                      double2* r64, float2* r32, int nrhs, double* part, int* nblk_out, const CgScalars* cgs);
// y = A x; if part != nullptr, per-block partial sums of ||D^dag x||^2 are written to
// part[k * nblk + b] and *nblk_out receives nblk.
// cgs (may be null): right-hand sides whose cgs[k].active is 0 are skipped. With pnew set,
// the operand is p = x + cgs[k].beta * pold, written to pnew for every site, and y = A p.
template <typename R>
int launch_apply_A(hmc_ctx* ctx, const Lat& lat, const R* phi, const cplx<R>* x, cplx<R>* y,
                   int nrhs, double* part, int* nblk_out, const CgScalars* cgs = nullptr,
                   const cplx<R>* pold = nullptr, cplx<R>* pnew = nullptr);
// strip.cu: the complex64 plain operator on full-height strips (L a multiple of 16 up to 80);
// same contract as launch_apply_A without the direction update. part_q (may be null): partial
// sums of ||A x||^2, laid out like part.
bool strip_supported(const Lat& lat);
int launch_apply_A_strip(hmc_ctx* ctx, const Lat& lat, const float* phi, const float2* x, float2* y, int nrhs,
                         double* part, int* nblk_out, const CgScalars* cgs, double* part_q = nullptr);
// fermion (+ boson) force and the action pieces, see force() in hmc.h. Y (may be null): D^dagger X
// already computed (same layout as X); otherwise the kernel forms it.
int launch_force(hmc_ctx* ctx, const Lat& lat, double r, const double* phi, const double2* X,
                 const double2* pf, int nrhs, double* F, int include_boson, double* part,
                 int* nblk_out, const double2* Y = nullptr);
int launch_boson(hmc_ctx* ctx, const Lat& lat, double r, const double* phi, double* F,
                 double* part, int* nblk_out);

// fft.cu
FftPlan* get_plan(hmc_ctx* ctx, int n);
int build_plans(hmc_ctx* ctx);
void free_plans(hmc_ctx* ctx);
// unitary FFT of complex data viewed as [outer][n][inner] along the middle axis, in place
// (src == nullptr) or from src into data; dir = -1 forward (e^{-2 pi i}), +1 inverse.
// cgs (may be null) with opr = outer indices per right-hand side: lines of inactive RHS are
// neither read nor written.
template <typename R>
int fft_axis(hmc_ctx* ctx, cplx<R>* data, int64_t outer, int n, int64_t inner, int dir,
             const cplx<R>* src = nullptr, const CgScalars* cgs = nullptr, int64_t opr = 1);
template <typename R>
// scratch (a vector's worth, aliasing neither x nor y): holds the complex64 (x, y) spectrum
// between the passes; without it the FP32 path takes the axis-by-axis kernels, which run in place
int launch_precond(hmc_ctx* ctx, const Lat& lat, const cplx<R>* x, cplx<R>* y, int nrhs, cplx<R>* scratch = nullptr);
// x += alpha p, r -= alpha q, z = P r for every active RHS with partial sums of ||r||^2 and
// <r, z> (rows of *nblk_out entries per RHS in part_r2, of *nblk_rz_out in part_rz).
template <typename R>
int launch_cg_update_precond(hmc_ctx* ctx, const Lat& lat, cplx<R>* x, cplx<R>* r, const cplx<R>* p,
                             const cplx<R>* q, cplx<R>* z, int nrhs, const CgScalars* cgs, double* part_r2,
                             double* part_rz, int* nblk_out, int* nblk_rz_out);
// complex64 PCG with the fused (x, y) passes (lattices where pcg_xy_path holds). One iteration
// after q = A p: launch_pcg_xy_forward does x += alpha p, r -= alpha q (partial ||r||^2), zhat
// = P-hat F~^* r in digit-permuted order (partial <r, z>); after beta, launch_pcg_xy_inverse
// forms the next direction pnew = F~ zhat + beta pold = z + beta pold.
bool pcg_xy_path(hmc_ctx* ctx, const Lat& lat);
int launch_pcg_xy_forward(hmc_ctx* ctx, const Lat& lat, float2* x, float2* r, const float2* p, const float2* q,
                          float2* zhat, int nrhs, const CgScalars* cgs, double* part_r2, double* part_rz,
                          int* nblk_r2, int* nblk_rz);
int launch_pcg_xy_inverse(hmc_ctx* ctx, const Lat& lat, const float2* zhat, const float2* pold, float2* pnew,
                          int nrhs, const CgScalars* cgs);
int metric_op(hmc_ctx* ctx, const Lat& lat, int op, const double* sig, const double* in,
              double* out, double eps, double* scalar_dev);

// randomized diagonal estimator of F~^* D^{-1} F~ over nrhs probes (fft.cu)
int green_run(hmc_ctx* ctx, int chain, const double* phi, const double2* v, int nrhs, double2* out, int precond,
              hmc_cg_stats* st);

// bounds build: per-translation-unit device error words (0 in the normal build)
unsigned int bounds_take_stencil();
unsigned int bounds_take_strip();

// batch.cu: all (chain, RHS) pairs of the context solve A X = b in one persistent launch (mixed
// precision, no preconditioner). b, x: concatenated [chain][k][V][4] complex128.
// batch_alloc (hmc_init) allocates the workspace for nrhs_max; batched_begin builds the tile
// table for K right-hand sides and uploads the chain table (phi pointers) of a trajectory;
// batched_solve enqueues one solve of every pair from b into x (from x when use_x0) and records
// its statistics in slot `slot` on the device, with no host synchronisation (so it can be
// captured in a CUDA graph); batched_collect reads the statistics of solves [0, nsolves) back: per
// solve and chain the iterations of its slowest pair and its worst true relative residual, per
// solve the reliable updates.
int batch_alloc(hmc_ctx* ctx);
int batched_begin(hmc_ctx* ctx, int K, const double* const* phi);
int batched_solve(hmc_ctx* ctx, int K, const double2* b, double2* x, bool use_x0, double tol, int maxit, int slot);
int batched_collect(hmc_ctx* ctx, int K, int nsolves, int* iterations, double* worst_resid, int* reliable_updates);
void batch_free(hmc_ctx* ctx);

// device error word: reads it (synchronising the stream) and returns HMC_ERR_TIMEOUT, clearing
// it, if a bounded device-side wait gave up since the last check (hmc.cu)
int check_device_flags(hmc_ctx* ctx);

// reductions: sum nblk partials for each of k rows into out[k] (device)
int reduce_rows(hmc_ctx* ctx, const double* part, int k, int nblk, double* out);

// cg.cu; with use_x0 the solve starts from the contents of x instead of zero. y_ready (may be
// null): set when ctx->d_z64 holds D^dagger x of the returned solution, computed in FP64 by the
// true-residual evaluation that ended each right-hand side's solve (mixed mode).
int cg_run(hmc_ctx* ctx, int chain, const double* phi, const double2* b, double2* x, int nrhs,
           double tol, int maxit, int precond, hmc_cg_stats* st, bool use_x0 = false, bool* y_ready = nullptr);

}  // namespace hmc
